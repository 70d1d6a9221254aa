// Device-side declarations shared by the library's CUDA translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mlp.cuh"

namespace dgk {

// per-element geometry record (float64), 32 words = 256 bytes
constexpr int kGeoStride = 32;
constexpr int kGeoDrdx = 0;     // 9: d r_a / d x_b at a*3+b
constexpr int kGeoNrm = 9;      // 12: outward unit normal of face f at 9 + 3f
constexpr int kGeoFscale = 21;  // 4: sJ / J
constexpr int kGeoSJ = 25;      // 4: face area / 2
constexpr int kGeoJ = 29;       // 1: volume / (4/3)

// status bits latched by the kernels
constexpr int kStatusBadState = 1;
constexpr int kStatusTimeout = 2;   // a bounded wait for tensor-core completion gave up
constexpr int kStatusBounds = 4;    // a device bounds check failed (debug build)

// Device bounds checks of the debug build (compiled with -DDG_BOUNDS_CHECK):
// DG_IN(cond, status) is true where cond holds; where it does not, it
// latches kStatusBounds in *status and is false, and the caller skips the
// access it guards. In the release build it is the constant true and the
// compiler removes the test: the kernels' code is unchanged.
#ifdef DG_BOUNDS_CHECK
#define DG_IN(cond, status) ((cond) ? true : (atomicOr((status), ::dgk::kStatusBounds), false))
constexpr bool kBoundsChecked = true;
#else
#define DG_IN(cond, status) true
constexpr bool kBoundsChecked = false;
#endif

// face connection word: >= 0: (neighbour element << 5) | (neighbour face << 3) | orientation;
// < 0: boundary, id = -1 - word
__host__ __device__ inline int32_t conn_interior(int32_t e2, int f2, int o) {
  return (e2 << 5) | (f2 << 3) | o;
}

struct Gas {
  double gamma, gm1, rho0, p0, u0[3], c0, E0, s_inf;
};

// Boundary-flux ledger, advanced inside the stage kernels: every CTA writes
// the sum of its tiles' contributions (in its own fixed tile order) to
// part[blockIdx.x]; the CTA that takes the last ticket of the launch adds
// the partials in CTA order and advances ledger = [L(5), Lres(5)] by the
// same Runge-Kutta stage as the state (res = a res + dt f, L += b res).
// The ticket counter only grows, so it needs no reset between launches;
// every CTA of every launch takes exactly one ticket, and all launches of a
// context use the same grid.
struct LedgerArgs {
  double* part;                // [gridDim.x][5]
  double* ledger;              // [10]
  unsigned long long* ticket;  // monotone counter
  double a, b, dt;
  int update;                  // 0: leave the ledger alone (dg_eval_rhs)
};

// Called by every thread of every CTA after the tile loop; threads 0..4
// hold the CTA's sums. Needs at least 160 threads per CTA.
__device__ inline void ledger_finish(const LedgerArgs& L, double cta_sum) {
  __shared__ double s_sum[5];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  if (tid < 5) s_sum[tid] = cta_sum;
  __syncthreads();
  if (tid == 0) {
    for (int v = 0; v < 5; ++v) L.part[size_t(blockIdx.x) * 5 + v] = s_sum[v];
    __threadfence();
    s_last = ((atomicAdd(L.ticket, 1ull) + 1ull) % gridDim.x) == 0ull;
  }
  __syncthreads();
  if (s_last && tid < 160) {       // warp v adds variable v over the CTAs, in a fixed order
    __threadfence();
    const int v = tid >> 5, lane = tid & 31;
    double x = 0.0;
    for (unsigned b = lane; b < gridDim.x; b += 32) x += __ldcg(L.part + size_t(b) * 5 + v);
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0 && L.update) {
      const double r = (L.a != 0.0) ? L.a * L.ledger[5 + v] + L.dt * x : L.dt * x;
      L.ledger[5 + v] = r;
      L.ledger[v] += L.b * r;
    }
  }
}

struct StageArgs {
  const double* q_in;
  double* q_out;
  double* res;
  const double* geo;         // [K][kGeoStride]
  const int32_t* conn;       // [K][4]
  const double* ops;         // DrT | DsT | DtT ([j][i], Np*Np each) | LIFTT ([m][i], NF*Np) | face_w [NF]
  const uint8_t* nbr_tbl;    // [4][4][6][Nfp]: neighbour volume node; then the same
                             // shape: neighbour face node (index in its face's list)
  const int32_t* fmask;      // [4][Nfp]
  const uint8_t* face_list;  // [ntiles][16 + 4 ET rounded up to 16 B]: header, then (le << 2 | f)
  LedgerArgs led;
  int* status;
  int64_t K;
  int ntiles;
  int bc_mode[8];
  double a, b, dt;
  Gas gas;
  double inflow[3];          // mode 4 ghost at the stage time: rho, rho u_in, E
  int64_t K_all;             // elements of the local mesh (own and halo): bound of neighbour ids
  // the paper's discretisation (stage_modal.cu): Iq [Nq][Np] | Sv [3][Np][Nq] |
  // Ifn [4][7][Nfq][Nfp] | Sf [4][7][Np][Nfq] | wf [Nfq]; null for the nodal forms
  const double* modal_ops;
};

// Float32 perturbation-form stage (stage_f32.cu)
struct StageArgsF32 {
  const float* q_in;         // q' = q - q0, [K][5][Np]
  float* q_out;
  float* res;
  const float* geo;          // [K][kGeoStride] float32 copy of the geometry record
  const int32_t* conn;
  const float* ops;          // same packing as StageArgs::ops, float32
  const uint8_t* nbr_tbl;
  const int32_t* fmask;
  LedgerArgs led;
  int* status;
  int64_t K;
  int ntiles;
  int bc_mode[8];
  float a, b, dt;
  Gas gas;
  float inflow[3];           // mode 4 ghost at the stage time, perturbation form:
                             // rho - rho0, rho u_in, E - E0
  // learned closure (boundary mode 3): incoming-invariant increments
  // [boundary face slot][Nfp] from launch_closure, or null (characteristic)
  const float* bD;
  // per tile, a 16-byte header (int32 total, inside the tile, to other
  // tiles, 0) then the faces it evaluates, one byte each (element in tile
  // << 2 | face), in that order: faces between two elements of the tile
  // (once, under the lower element), faces to other tiles, outer faces
  const uint8_t* face_list;  // [ntiles][16 + 4 ET rounded up to 16 B]
  int64_t K_all;             // elements of the local mesh (own and halo): bound of neighbour ids
  int64_t nb;                // boundary face slots (rows of bD)
  // launched as a programmatic dependent of the kernel before it in the
  // stream (the closure, which writes bD): every CTA stages its operators and
  // starts its first tile's copies, then waits for that kernel (griddep_wait)
  int pdl;
};

// Programmatic dependent launch (sm_90 and later). A kernel launched with
// launch_stage_kernel(..., pdl = true) may start while the kernel before it
// in the stream still runs, once every CTA of that kernel has executed
// griddep_launch_dependents (or exited); griddep_wait returns when that
// kernel has completed and its memory operations are visible. Without a
// programmatic predecessor both are no-ops.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename T>
inline cudaError_t launch_stage_kernel(void (*k)(T), int grid, int threads, size_t smem,
                                       cudaStream_t s, const T& a, bool pdl) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(threads));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, a);
}

int stage_f32_tile_elems(int p);
cudaError_t stage_f32_prepare(int p, int* blocks_per_sm);
cudaError_t launch_stage_f32(int p, const StageArgsF32& a, int grid, cudaStream_t s);
cudaError_t launch_to_perturbation(const double* q, float* qp, int64_t K, int Np, double rho0,
                                   double E0, cudaStream_t s);
cudaError_t launch_from_perturbation(const float* qp, double* q, int64_t K, int Np, double rho0,
                                     double E0, cudaStream_t s);
cudaError_t launch_widen(const float* x, double* y, int64_t n, cudaStream_t s);
cudaError_t launch_probe_sample_f32(const float* q, int Np, int n, const int32_t* elem,
                                    const double* rows, double rho0, double E0, double* out,
                                    cudaStream_t s);

// Tensor-core form of the float32 stage (stage_tc.cu), orders 1..4; uses
// StageArgsF32 with ops pointing at the image built by build_tc_ops.
// images = 2: tf32 head and tail of both operands, three MMAs per k-step
// (DG_PREC_F32_TC); images = 1: one MMA per k-step on the float32 values
// read as tf32 (DG_PREC_F32_TC1).
size_t stage_tc_ops_bytes(int p, int images);
int stage_tc_tile_elems(int p);
int stage_tc_ctas_per_sm(int p);
void build_tc_ops(int p, int images, const double* Dr, const double* Ds, const double* Dt,
                  const double* LIFT, const double* face_w, unsigned char* out);
cudaError_t stage_tc_prepare(int p, int images, int* blocks_per_sm);
cudaError_t launch_stage_tc(int p, int images, const StageArgsF32& a, int grid, cudaStream_t s);

// Learned closure (learned.cu)
struct BaseGhost;
cudaError_t launch_sample_traces(const float* q, int Np, int Nfp, const int32_t* tr_elem,
                                 const int8_t* tr_face, const int32_t* conn, const uint8_t* tbl,
                                 const int32_t* fmask, const float* geo, const float* txyz,
                                 const float* tr_psi, int64_t n, const BaseGhost& bg,
                                 const mlp::Scales& S, float* X, float* Y, float* amp, int* status,
                                 cudaStream_t s);
// Per Runge-Kutta stage, before the stage kernel: at every node of the
// boundary faces whose id has mode 3, the increment D of the incoming
// invariant from the network (D = 0 without one) and, when `advance`, the
// memory's 2N-storage update res = a res + dt dpsi/dt, psi += b res.
struct ClosureArgs {
  const float* q;            // stage input, perturbation form [K][5][Np]
  int Np, Nfp;
  const int32_t* bface;      // [nb] e * 4 + f of every boundary face, slot order
  int64_t nb;
  const int32_t* conn;
  const int32_t* fmask;
  const float* geo;
  const float* bxyz;         // [nb][Nfp][3]
  int bc_mode[8];
  const float* w;            // network parameters or null
  const unsigned char* wimg; // their operand image (launch_closure_image), with w
  mlp::Scales S;
  float* psi;                // [nb][Nfp] memory
  float* psi_res;
  float* D;                  // [nb][Nfp] out
  float a, b, dt;
  int advance;
  int* status;               // kStatusTimeout when a tensor-core completion wait gives up
  int64_t K_all;             // elements of the local mesh: bound of bface's element ids
};
cudaError_t launch_closure(const ClosureArgs& A, const BaseGhost& bg, cudaStream_t s);
// shared-memory attributes of the closure kernel on the current device
cudaError_t closure_prepare();
// The closure's weight image (operand layouts of W1 and W2 as tf32 head and
// tail, and the vectors it reads) from the parameter vector; rebuild after
// every change of the parameters.
size_t closure_image_bytes();
cudaError_t launch_closure_image(const float* w, unsigned char* img, cudaStream_t s);
// The same memory at the nodes of the trace faces (inner traces), advanced
// per stage while traces are recorded.
cudaError_t launch_trace_memory(const float* q, int Np, int Nfp, const int32_t* tr_elem,
                                const int8_t* tr_face, const int32_t* fmask, const float* geo,
                                const float* txyz, int64_t n, const BaseGhost& bg,
                                const mlp::Scales& S, float* psi, float* psi_res, float a,
                                float b, float dt, cudaStream_t s);
int mlp_grad_blocks(int64_t N, int sms);
// shared-memory attribute of the training kernel on the current device
cudaError_t mlp_prepare();
cudaError_t launch_mlp_loss_grad(const float* w, const float* X, const float* Y, int64_t N,
                                 int nblocks, float* part_grad, float* part_loss, float* grad,
                                 double* loss, cudaStream_t s);
cudaError_t launch_adam(float* w, const float* grad, float* m, float* v, float lr, int t,
                        cudaStream_t s);
cudaError_t launch_mlp_forward(const float* w, const float* X, int64_t N, float* out,
                               cudaStream_t s);

// launch helpers (stage_fp64.cu)
int stage_tile_elems(int p);
size_t stage_smem_bytes(int p);
cudaError_t stage_prepare(int p, int* blocks_per_sm);
cudaError_t launch_stage(int p, const StageArgs& a, int grid, cudaStream_t s);
// The paper's discretisation (stage_modal.cu); modal_ops_len: doubles of the operator block
int stage_modal_tile_elems(int p);
int modal_ops_len(int p);
cudaError_t stage_modal_prepare(int p, int* blocks_per_sm);
cudaError_t launch_stage_modal(int p, const StageArgs& a, int grid, cudaStream_t s);

cudaError_t launch_probe_sample(const double* q, int Np, int n, const int32_t* elem,
                                const double* rows, double* out, cudaStream_t s);
// halo exchange of a partitioned mesh (halo.cu): entries ef[i] = e * 4 + f,
// buffers [n][5][Nfp] of the state's type
template <typename T>
cudaError_t launch_halo_pack(const T* q, int Np, int Nfp, const int32_t* ef, const int32_t* fmask,
                             int64_t n, T* buf, int64_t K_all, int* status, cudaStream_t s);
template <typename T>
cudaError_t launch_halo_unpack(T* q, int Np, int Nfp, const int32_t* ef, const int32_t* fmask,
                               int64_t n, const T* buf, int64_t K_all, int* status, cudaStream_t s);
cudaError_t launch_totals(const double* q, const double* geo, const double* mass_w, int64_t K,
                          int Np, double* partial, int nblocks, double* out, cudaStream_t s);

}  // namespace dgk
