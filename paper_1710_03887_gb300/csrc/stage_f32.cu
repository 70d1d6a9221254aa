// Float32 perturbation form of the Runge-Kutta stage (the precision form of
// the method): the state is stored as q' = q - q0 relative to the resting
// free stream q0 = (rho0, 0, 0, 0, E0), so the pressure
//   p' = (gamma-1) (E' - |m'|^2 / (2 rho))            (Eq. 2 minus its base value)
// carries no cancellation against p0, and every flux is formed minus the
// constant base flux (whose divergence and jump vanish):
//   F'_d = (m'_d, m'_1 u_d + p' delta_1d, m'_2 u_d + p' delta_2d,
//           m'_3 u_d + p' delta_3d, u_d (H0 + E' + p')),  H0 = E0 + p0.
// The LLF jump in this form is
//   n.F(q-) - F* = ((n.F')(q'-) - (n.F')(q'+)) / 2 + lambda (q'+ - q'-) / 2,
// and outer-face ghost states follow the same rules as the float64 path,
// rewritten in perturbation quantities (ghost_state_f). Fused like the
// float64 kernel: one launch per stage, operators in shared memory, every
// face evaluated from both sides, no atomics; GB300's float64 pipe is left
// idle except for the per-tile boundary-flux sums.
#include <cmath>

#include "dg_device.cuh"
#include "ghost_f32.cuh"

namespace dgk {

template <int P>
struct OrderF {
  static constexpr int Np = (P + 1) * (P + 2) * (P + 3) / 6;
  static constexpr int Nfp = (P + 1) * (P + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int ET = P == 1 ? 64 : P == 2 ? 32 : P == 3 ? 16 : 8;
  static constexpr int NT = (ET * Np + 31) / 32 * 32;
  static constexpr int kOps = 3 * Np * Np + NF * Np + NF;
  static constexpr int kTbl = 4 * 4 * 6 * Nfp;
  // shared memory, in floats
  static constexpr int oOps = 0;
  static constexpr int oQ = oOps + kOps;
  static constexpr int oF = oQ + ET * 5 * Np;
  static constexpr int oDF = oF + ET * 15 * Np;
  static constexpr int oGeo = oDF + ET * 5 * NF;
  static constexpr int oEnd = oGeo + ET * kGeoStride;
  static constexpr int nWarps = NT / 32;
  // doubles for the ledger reduction, then integers
  static constexpr size_t oRedB = (size_t(oEnd) * 4 + 15) / 16 * 16;
  static constexpr size_t oConnB = oRedB + size_t(nWarps) * 5 * 8;
  static constexpr size_t oFmaskB = oConnB + size_t(ET) * 4 * 4;
  static constexpr size_t oTblB = oFmaskB + size_t(4) * Nfp * 4;
  static constexpr size_t bytes = (oTblB + kTbl + 15) / 16 * 16;
};

struct BaseF {
  float rho0, p0, gamma, gm1, H0;
};

// velocity, pressure perturbation and 1/rho of a perturbation state
__device__ __forceinline__ void prim_f(const float q[5], const BaseF& b, float& rinv, float u[3],
                                       float& pp) {
  rinv = 1.0f / (b.rho0 + q[0]);
  u[0] = q[1] * rinv;
  u[1] = q[2] * rinv;
  u[2] = q[3] * rinv;
  pp = b.gm1 * (q[4] - 0.5f * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
}

// (n.F)' and |u.n| + c of a perturbation state
__device__ __forceinline__ void normal_flux_f(const float q[5], const float n[3], const BaseF& b,
                                              float fn[5], float& lam) {
  float rinv, u[3], pp;
  prim_f(q, b, rinv, u, pp);
  const float un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  fn[0] = q[1] * n[0] + q[2] * n[1] + q[3] * n[2];
  fn[1] = q[1] * un + pp * n[0];
  fn[2] = q[2] * un + pp * n[1];
  fn[3] = q[3] * un + pp * n[2];
  fn[4] = un * (b.H0 + q[4] + pp);
  lam = fabsf(un) + sqrtf(b.gamma * (b.p0 + pp) * rinv);
}

template <int P>
__global__ void __launch_bounds__(OrderF<P>::NT)
stage_f32_kernel(const StageArgsF32 A) {
  using O = OrderF<P>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF, ET = O::ET, NT = O::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  float* sOps = sm + O::oOps;
  float* sQ = sm + O::oQ;
  float* sF = sm + O::oF;
  float* sDF = sm + O::oDF;
  float* sGeo = sm + O::oGeo;
  double* sRed = reinterpret_cast<double*>(smem_raw + O::oRedB);
  int32_t* sConn = reinterpret_cast<int32_t*>(smem_raw + O::oConnB);
  int32_t* sFmask = reinterpret_cast<int32_t*>(smem_raw + O::oFmaskB);
  uint8_t* sTbl = smem_raw + O::oTblB;
  const float* DrT = sOps;
  const float* DsT = sOps + Np * Np;
  const float* DtT = sOps + 2 * Np * Np;
  const float* LiftT = sOps + 3 * Np * Np;
  const float* faceW = LiftT + NF * Np;
  const int tid = threadIdx.x;

  for (int i = tid; i < O::kOps; i += NT) sOps[i] = A.ops[i];
  for (int i = tid; i < O::kTbl; i += NT) sTbl[i] = A.nbr_tbl[i];
  for (int i = tid; i < 4 * Nfp; i += NT) sFmask[i] = A.fmask[i];
  const BaseF b{float(A.gas.rho0), float(A.gas.p0), float(A.gas.gamma), float(A.gas.gm1),
                float(A.gas.E0 + A.gas.p0)};
  const BaseGhost bg{float(A.gas.rho0), float(A.gas.p0), float(A.gas.gamma), float(A.gas.gm1),
                     float(A.gas.c0)};

  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
    const int64_t e0 = int64_t(tile) * ET;
    const int nE = int((A.K - e0) < ET ? (A.K - e0) : int64_t(ET));
    __syncthreads();
    {
      const float* gq = A.q_in + e0 * 5 * Np;
      for (int i = tid; i < nE * 5 * Np; i += NT) sQ[i] = gq[i];
      const float* gg = A.geo + e0 * kGeoStride;
      for (int i = tid; i < nE * kGeoStride; i += NT) sGeo[i] = gg[i];
      const int32_t* gc = A.conn + e0 * 4;
      for (int i = tid; i < nE * 4; i += NT) sConn[i] = gc[i];
    }
    __syncthreads();

    // ---- volume fluxes (perturbation form) at nodes
    {
      const int le = tid / Np, n = tid - (tid / Np) * Np;
      if (le < nE) {
        float q[5];
        for (int v = 0; v < 5; ++v) q[v] = sQ[(le * 5 + v) * Np + n];
        float rinv, u[3], pp;
        prim_f(q, b, rinv, u, pp);
        if (!(b.rho0 + q[0] > 0.0f) || !(b.p0 + pp > 0.0f) || !isfinite(q[4]) || !isfinite(pp))
          atomicOr(A.status, kStatusBadState);
        const float H = b.H0 + q[4] + pp;
        float F[3][5];
        for (int d = 0; d < 3; ++d) {
          F[d][0] = q[1 + d];
          F[d][1] = q[1] * u[d];
          F[d][2] = q[2] * u[d];
          F[d][3] = q[3] * u[d];
          F[d][1 + d] += pp;
          F[d][4] = u[d] * H;
        }
        const float* dr = sGeo + le * kGeoStride + kGeoDrdx;
        for (int a = 0; a < 3; ++a) {
          const float m0 = dr[a * 3], m1 = dr[a * 3 + 1], m2 = dr[a * 3 + 2];
          for (int v = 0; v < 5; ++v)
            sF[(le * 15 + a * 5 + v) * Np + n] = m0 * F[0][v] + m1 * F[1][v] + m2 * F[2][v];
        }
      }
    }

    // ---- face fluxes at face nodes
    float led[5] = {0, 0, 0, 0, 0};   // float32 within the tile, float64 across tiles
    bool any_bdry = false;
    for (int it = tid; it < nE * NF; it += NT) {
      const int le = it / NF, fm = it - (it / NF) * NF;
      const int f = fm / Nfp, m = fm - (fm / Nfp) * Nfp;
      const int n = sFmask[f * Nfp + m];
      float qm[5], qp[5];
      for (int v = 0; v < 5; ++v) qm[v] = sQ[(le * 5 + v) * Np + n];
      const float* geo = sGeo + le * kGeoStride;
      const float nv[3] = {geo[kGeoNrm + 3 * f], geo[kGeoNrm + 3 * f + 1], geo[kGeoNrm + 3 * f + 2]};
      const int32_t c = sConn[le * 4 + f];
      if (c >= 0) {
        const int64_t e2 = c >> 5;
        const int f2 = (c >> 3) & 3, o = c & 7;
        const int n2 = sTbl[((f * 4 + f2) * 6 + o) * Nfp + m];
        const float* src = A.q_in + e2 * 5 * Np + n2;
        for (int v = 0; v < 5; ++v) qp[v] = __ldg(src + v * Np);
      } else {
        const int mode = A.bc_mode[(-1 - c) & 7];
        if (mode == 3) {
          const float D = A.bD ? A.bD[size_t((-1 - c) >> 3) * Nfp + m] : 0.0f;
          ghost_learned_f(qm, nv, bg, D, qp);
        } else {
          ghost_state_f(mode, qm, nv, bg, qp);
        }
      }
      float fnm[5], fnp[5], lm, lp;
      normal_flux_f(qm, nv, b, fnm, lm);
      normal_flux_f(qp, nv, b, fnp, lp);
      const float lam = fmaxf(lm, lp);
      const float fs = geo[kGeoFscale + f];
      for (int v = 0; v < 5; ++v) {
        const float jump = 0.5f * (fnm[v] - fnp[v]) + 0.5f * lam * (qp[v] - qm[v]);
        sDF[(le * 5 + v) * NF + fm] = fs * jump;
        if (c < 0) {
          const float fstar = 0.5f * (fnm[v] + fnp[v]) - 0.5f * lam * (qp[v] - qm[v]);
          led[v] += faceW[fm] * geo[kGeoSJ + f] * fstar;
        }
      }
      any_bdry |= (c < 0);
    }
    if (__syncthreads_or(any_bdry)) {
      const int lane = tid & 31, warp = tid >> 5;
      for (int v = 0; v < 5; ++v) {
        float x = led[v];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) sRed[warp * 5 + v] = double(x);
      }
      __syncthreads();
      if (tid < 5) {
        double acc = 0.0;
        for (int w = 0; w < O::nWarps; ++w) acc += sRed[w * 5 + tid];
        const int slot = A.ledger_slot[tile];
        if (slot >= 0) A.ledger_part[size_t(slot) * 5 + tid] = acc;
      }
    }
    __syncthreads();

    // ---- per node: contraction, lift, Runge-Kutta update
    {
      const int le = tid / Np, n = tid - (tid / Np) * Np;
      if (le < nE) {
        float acc[5] = {0, 0, 0, 0, 0};
        const float* Fr = sF + (le * 15) * Np;
        const float* Fs = Fr + 5 * Np;
        const float* Ft = Fr + 10 * Np;
#pragma unroll 4
        for (int j = 0; j < Np; ++j) {
          const float dr = DrT[j * Np + n], ds = DsT[j * Np + n], dt = DtT[j * Np + n];
#pragma unroll
          for (int v = 0; v < 5; ++v)
            acc[v] += dr * Fr[v * Np + j] + ds * Fs[v * Np + j] + dt * Ft[v * Np + j];
        }
        float out[5];
        for (int v = 0; v < 5; ++v) out[v] = -acc[v];
        const float* dF = sDF + (le * 5) * NF;
#pragma unroll 4
        for (int m = 0; m < NF; ++m) {
          const float l = LiftT[m * Np + n];
#pragma unroll
          for (int v = 0; v < 5; ++v) out[v] += l * dF[v * NF + m];
        }
        const int64_t base = (e0 + le) * 5 * Np + n;
        for (int v = 0; v < 5; ++v) {
          const int64_t ix = base + int64_t(v) * Np;
          const float r = (A.a != 0.0f) ? A.a * A.res[ix] + A.dt * out[v] : A.dt * out[v];
          A.res[ix] = r;
          A.q_out[ix] = sQ[(le * 5 + v) * Np + n] + A.b * r;
        }
      }
    }
  }
}

int stage_f32_tile_elems(int p) {
  switch (p) {
    case 1: return OrderF<1>::ET;
    case 2: return OrderF<2>::ET;
    case 3: return OrderF<3>::ET;
    default: return OrderF<4>::ET;
  }
}

template <int P>
static cudaError_t prepare_f32_impl(int* bps) {
  cudaError_t e = cudaFuncSetAttribute(stage_f32_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(OrderF<P>::bytes));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, stage_f32_kernel<P>, OrderF<P>::NT,
                                                       OrderF<P>::bytes);
}

cudaError_t stage_f32_prepare(int p, int* bps) {
  switch (p) {
    case 1: return prepare_f32_impl<1>(bps);
    case 2: return prepare_f32_impl<2>(bps);
    case 3: return prepare_f32_impl<3>(bps);
    default: return prepare_f32_impl<4>(bps);
  }
}

cudaError_t launch_stage_f32(int p, const StageArgsF32& a, int grid, cudaStream_t s) {
  switch (p) {
    case 1: stage_f32_kernel<1><<<grid, OrderF<1>::NT, OrderF<1>::bytes, s>>>(a); break;
    case 2: stage_f32_kernel<2><<<grid, OrderF<2>::NT, OrderF<2>::bytes, s>>>(a); break;
    case 3: stage_f32_kernel<3><<<grid, OrderF<3>::NT, OrderF<3>::bytes, s>>>(a); break;
    default: stage_f32_kernel<4><<<grid, OrderF<4>::NT, OrderF<4>::bytes, s>>>(a); break;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------- conversions, etc.

// q' = float(q - q0) and back, per variable
__global__ void to_perturbation_kernel(const double* q, float* qp, int64_t n_rows, int Np,
                                       double rho0, double E0) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_rows * Np) return;
  const int v = int((i / Np) % 5);
  const double base = v == 0 ? rho0 : (v == 4 ? E0 : 0.0);
  qp[i] = float(q[i] - base);
}

__global__ void from_perturbation_kernel(const float* qp, double* q, int64_t n_rows, int Np,
                                         double rho0, double E0) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_rows * Np) return;
  const int v = int((i / Np) % 5);
  const double base = v == 0 ? rho0 : (v == 4 ? E0 : 0.0);
  q[i] = base + double(qp[i]);
}

__global__ void widen_kernel(const float* x, double* y, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) y[i] = double(x[i]);
}

cudaError_t launch_to_perturbation(const double* q, float* qp, int64_t K, int Np, double rho0,
                                   double E0, cudaStream_t s) {
  const int64_t n = K * 5 * Np;
  to_perturbation_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(q, qp, K * 5, Np, rho0, E0);
  return cudaGetLastError();
}

cudaError_t launch_from_perturbation(const float* qp, double* q, int64_t K, int Np, double rho0,
                                     double E0, cudaStream_t s) {
  const int64_t n = K * 5 * Np;
  from_perturbation_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(qp, q, K * 5, Np, rho0, E0);
  return cudaGetLastError();
}

cudaError_t launch_widen(const float* x, double* y, int64_t n, cudaStream_t s) {
  widen_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

}  // namespace dgk

namespace dgk {

// Sensor values of the float32 perturbation state, returned as total state:
// out[probe][v] = q0_v + sum_n row[probe][n] q'[elem][v][n]
__global__ void probe_f32_kernel(const float* q, int Np, int n, const int32_t* elem,
                                 const double* rows, double rho0, double E0, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * 5) return;
  const int pidx = i / 5, v = i - (i / 5) * 5;
  const float* src = q + (int64_t(elem[pidx]) * 5 + v) * Np;
  const double* row = rows + size_t(pidx) * Np;
  double acc = 0.0;
  for (int j = 0; j < Np; ++j) acc += row[j] * double(src[j]);
  out[i] = (v == 0 ? rho0 : (v == 4 ? E0 : 0.0)) + acc;
}

cudaError_t launch_probe_sample_f32(const float* q, int Np, int n, const int32_t* elem,
                                    const double* rows, double rho0, double E0, double* out,
                                    cudaStream_t s) {
  const int threads = 128, blocks = (n * 5 + threads - 1) / threads;
  probe_f32_kernel<<<blocks, threads, 0, s>>>(q, Np, n, elem, rows, rho0, E0, out);
  return cudaGetLastError();
}

}  // namespace dgk
