// Tensor-core form of the float32 perturbation stage (DG_PREC_F32_TC).
//
// Same arithmetic as stage_f32.cu up to the two contractions, which become
// one dense GEMM per tile of 12 elements on the tcgen05 tensor cores:
//
//   rhs[(e,v), i] = sum_k A[(e,v), k] B[i, k]
//   A[(e,v), :] = [ Fr'_v(e, 0..Np) | Fs'_v | Ft'_v | dF_v(e, 0..4Nfp) ]     (M = 64 rows)
//   B[i, :]     = [ -Dr[i, :] | -Ds[i, :] | -Dt[i, :] | LIFT[i, :] ]       (N = Np padded to 8)
//
// i.e. the volume term and the surface lift of Eq. 10 in one contraction of
// length K = 3 Np + 4 Nfp. Both operands are split into a tf32 head and a
// tf32 tail (x = hi + lo) and the product is formed as
// A_hi B_hi + A_hi B_lo + A_lo B_hi in float32 accumulators in tensor memory,
// which keeps float32-level accuracy (the dropped lo*lo term is ~2^-22).
//
// The node and face phases write every A entry as float32 straight into the
// MMA operand layout of the head image (no row-major staging copy of A); the
// node phase maps a warp onto 8 elements x 4 nodes so that its stores land
// on 32 different banks. One linear pass over that image then splits each
// 16-byte chunk in place into head and tail (the tail into the second
// image), whatever rows and columns the chunk holds. A tile needs ~104 KB
// of shared memory at p = 3, so two CTAs share an SM and one computes while
// the other waits at a barrier or on its MMAs; at p = 4 (~183 KB: the
// operand images alone are ~140 KB) one CTA of 512 threads takes the SM. The accumulator rows come
// back from tensor memory into a small staging array and the Runge-Kutta
// update runs coalesced over the tile's state.
#include <cmath>
#include <cstring>

#include "cp_async.cuh"
#include "dg_device.cuh"
#include "ghost_f32.cuh"
#include "tc_ptx.cuh"

namespace dgk {

// S = operand images per operand: 2 (tf32 head and tail, three MMAs per
// k-step: the float32-level form) or 1 (the float32 values read as tf32 by
// the MMA, one MMA per k-step: the one-pass variant, DG_PREC_F32_TC1)
template <int P, int S = 2>
struct OrderTC {
  static constexpr int Np = (P + 1) * (P + 2) * (P + 3) / 6;
  static constexpr int Nfp = (P + 1) * (P + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int ET = 12;                        // 60 of the 64 MMA rows
  static constexpr int M = 64;
  static constexpr int N = (Np + 7) / 8 * 8;           // M = 64: N a multiple of 8
  static constexpr int KU = 3 * Np + NF;               // used columns
  static constexpr int K = (KU + 7) / 8 * 8;
  // p <= 3: two CTAs of 256 threads per SM (~104 KB of shared memory each at
  // p = 3); p = 4: the operands alone take ~140 KB, one CTA of 512 threads
  static constexpr int CPS = P <= 3 ? 2 : 1;
  static constexpr int NT = P <= 3 ? 256 : 512;
  static constexpr uint32_t TCOLS = N <= 32 ? 32u : 64u;   // tensor-memory columns (power of 2)
  static constexpr int NB = (Np + 3) / 4;              // node blocks of the node phase
  static constexpr int EG = (ET + 7) / 8;              // element groups of the node phase
  static constexpr int SO = Np % 2 ? Np : Np + 1;      // odd row stride of the results
  static constexpr int kQT = ET * 5 * Np;
  static constexpr int kG = ET * NF;                   // gathered traces per variable
  static constexpr uint32_t SBO = uint32_t(K / 4) * 128u;
  static constexpr uint32_t kABytes = uint32_t(M / 8) * SBO;
  static constexpr uint32_t kBBytes = uint32_t(N / 8) * SBO;
  // shared memory (bytes): A_hi, A_lo, B_hi, B_lo (operand layouts),
  // gathered neighbour traces [v][le NF + fm], results [row][SO], two
  // buffers of state, geometry and connections, face weights, reduction
  // space, tables, face lists, barrier
  static constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }
  static constexpr size_t oAhi = 0;
  static constexpr size_t oAlo = oAhi + kABytes;                   // (S = 2 only)
  static constexpr size_t oBhi = oAhi + size_t(S) * kABytes;
  static constexpr size_t oBlo = oBhi + kBBytes;                   // (S = 2 only)
  static constexpr size_t oG = al16(oBhi + size_t(S) * kBBytes);
  static constexpr size_t oR = al16(oG + size_t(5 * kG) * 4);
  static constexpr size_t oQ = al16(oR + size_t(5 * ET) * SO * 4);
  static constexpr size_t oGeo = al16(oQ + 2 * size_t(kQT) * 4);
  static constexpr size_t oW = al16(oGeo + 2 * size_t(ET) * kGeoStride * 4);
  static constexpr size_t oRed = al16(oW + size_t(NF) * 4);          // 8 warps x 5 doubles
  static constexpr size_t oConn = oRed + (NT / 32) * 5 * 8;          // 2 x ET*4 ints
  static constexpr size_t oFmask = oConn + 2 * size_t(ET) * 16;      // 4*Nfp ints
  static constexpr size_t oTbl = oFmask + size_t(NF) * 4;            // 2 x 96*Nfp bytes
  static constexpr size_t kFL = 16 + (4 * size_t(ET) + 15) / 16 * 16;   // face list row (16-byte multiple)
  static_assert(kFL % 16 == 0, "face-list rows are copied in 16-byte pieces");
  static constexpr size_t oFL = al16(oTbl + 2 * 96 * Nfp);           // 2 face-list buffers
  static constexpr size_t oBar = al16(oFL + 2 * kFL);                // mbarrier, tmem slot, flag
  static constexpr size_t bytes = oBar + 32;
  static_assert(bytes <= (CPS == 2 ? 113 : 227) * 1024, "CTAs per SM");
  static_assert(N <= 64, "accumulator rows read as 32 + 8 columns");
  static constexpr size_t kOpsBytes = S * size_t(kBBytes) + size_t(NF) * 4;   // B images + face weights
};

struct BaseF2 {
  float rho0, p0, gamma, gm1, H0, c0;
};

__device__ __forceinline__ void prim_tc(const float q[5], const BaseF2& b, float& rinv, float u[3],
                                        float& pp) {
  rinv = __fdividef(1.0f, b.rho0 + q[0]);          // 2 ulp: far below the form's tolerance
  u[0] = q[1] * rinv;
  u[1] = q[2] * rinv;
  u[2] = q[3] * rinv;
  pp = b.gm1 * (q[4] - 0.5f * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
}

__device__ __forceinline__ void normal_flux_tc(const float q[5], const float n[3], const BaseF2& b,
                                               float fn[5], float& lam) {
  float rinv, u[3], pp;
  prim_tc(q, b, rinv, u, pp);
  const float un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  fn[0] = q[1] * n[0] + q[2] * n[1] + q[3] * n[2];
  fn[1] = q[1] * un + pp * n[0];
  fn[2] = q[2] * un + pp * n[1];
  fn[3] = q[3] * un + pp * n[2];
  fn[4] = un * (b.H0 + q[4] + pp);
  const float c2 = b.gamma * (b.p0 + pp) * rinv;
  lam = fabsf(un) + (c2 > 0.0f ? c2 * rsqrtf(c2) : 0.0f);
}

// Parts of the LLF flux at a face node: n.F(q-), A = (n.F(q-) - n.F(q+)) / 2,
// B = lambda (q+ - q-) / 2; F* = n.F(q-) - A - B, the jump n.F(q-) - F* = A + B.
__device__ __forceinline__ void llf_parts_tc(const float qm[5], const float qp[5], const float n[3],
                                             const BaseF2& b, float fnm[5], float hA[5], float hB[5]) {
  float fnp[5], lm, lp;
  normal_flux_tc(qm, n, b, fnm, lm);
  normal_flux_tc(qp, n, b, fnp, lp);
  const float lam = fmaxf(lm, lp);
  for (int v = 0; v < 5; ++v) {
    hA[v] = 0.5f * (fnm[v] - fnp[v]);
    hB[v] = 0.5f * lam * (qp[v] - qm[v]);
  }
}

constexpr uint32_t kWaitTries = 1u << 24;   // bounded MMA completion wait
constexpr uint32_t kHintTries = 1u << 22;   // the same bound with a 200 ns suspend hint per try

// float32 value x into operand entry at byte offset off of the head image
// (split into head and tail later, chunk by chunk)
__device__ __forceinline__ void store_a(unsigned char* ahi, uint32_t off, float x) {
  *reinterpret_cast<float*>(ahi + off) = x;
}

// Per tile of 12 elements:
//  1. state, geometry, connections and face list arrived by cp.async during
//     the previous tile; neighbour traces of faces to other tiles are
//     gathered by cp.async into G while
//  2. the node phase writes the metric-folded fluxes into A (float32);
//  3. the face phase writes Fscale (n.F - F*) into the face columns of A (a
//     face between two elements of the tile once, both jumps);
//  4. every 16-byte chunk of A is split in place into its tf32 head and tail;
//  5. one thread issues the MMAs (A_hi B_hi + A_hi B_lo + A_lo B_hi, K/8
//     steps) and commits them to the mbarrier; the residuals load meanwhile;
//  6. warps 0..3 move their accumulator rows (M = 64: row r in tensor-memory
//     lane 32 (r / 16) + r % 16) into R, and all threads update q and res
//     with coalesced accesses.
template <int P, int S>
__global__ void __launch_bounds__(OrderTC<P, S>::NT, OrderTC<P, S>::CPS)
stage_tc_kernel(const StageArgsF32 A) {
  using O = OrderTC<P, S>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF, ET = O::ET, NT = O::NT;
  constexpr int K = O::K, SO = O::SO, kG = O::kG;
  constexpr uint32_t SBO = O::SBO;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* sAhi = smem + O::oAhi;
  [[maybe_unused]] unsigned char* sAlo = smem + O::oAlo;
  float* sG = reinterpret_cast<float*>(smem + O::oG);
  float* sR = reinterpret_cast<float*>(smem + O::oR);
  float* sW = reinterpret_cast<float*>(smem + O::oW);
  double* sRed = reinterpret_cast<double*>(smem + O::oRed);
  int32_t* sFmask = reinterpret_cast<int32_t*>(smem + O::oFmask);
  uint8_t* sTbl = smem + O::oTbl;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + O::oBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + O::oBar + 8);
  volatile int* sAbort = reinterpret_cast<volatile int*>(smem + O::oBar + 12);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // constant operand B (host-built images in the operand layout), face
  // weights, tables; A zeroed once (its padding rows and columns are never
  // written again and must stay finite)
  {
    const uint4* src = reinterpret_cast<const uint4*>(A.ops);
    uint4* dst = reinterpret_cast<uint4*>(smem + O::oBhi);
    for (int i = tid; i < int(S * O::kBBytes / 16); i += NT) dst[i] = src[i];
    uint4* a = reinterpret_cast<uint4*>(smem + O::oAhi);
    for (int i = tid; i < int(S * O::kABytes / 16); i += NT) a[i] = make_uint4(0, 0, 0, 0);
    const float* w = reinterpret_cast<const float*>(reinterpret_cast<const unsigned char*>(A.ops) +
                                                    S * O::kBBytes);
    for (int i = tid; i < NF; i += NT) sW[i] = w[i];
    for (int i = tid; i < 2 * 96 * Nfp; i += NT) sTbl[i] = A.nbr_tbl[i];   // volume- and face-node tables
    for (int i = tid; i < NF; i += NT) sFmask[i] = A.fmask[i];
  }
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sAbort = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, O::TCOLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const BaseF2 b{float(A.gas.rho0), float(A.gas.p0), float(A.gas.gamma), float(A.gas.gm1),
                 float(A.gas.E0 + A.gas.p0), float(A.gas.c0)};
  const BaseGhost bg{b.rho0, b.p0, b.gamma, b.gm1, b.c0, A.inflow[0], A.inflow[1], A.inflow[2]};
  constexpr uint32_t idesc = tc::idesc_tf32(O::M, O::N);
  uint32_t phase = 0;

  // asynchronous copy of tile t's state, geometry and connections into buffer bf
  auto prefetch = [&](int t, int bf) {
    if (t >= A.ntiles) return;
    const int64_t f0 = int64_t(t) * ET;
    const int n = int((A.K - f0) < ET ? (A.K - f0) : int64_t(ET));
    float* dq = reinterpret_cast<float*>(smem + O::oQ) + bf * O::kQT;
    const float* gq = A.q_in + f0 * 5 * Np;
    if constexpr ((5 * Np) % 4 == 0) {
      for (int i = tid; i < n * 5 * Np / 4; i += NT) cp_async16(dq + 4 * i, gq + 4 * i);
    } else {
      for (int i = tid; i < n * 5 * Np; i += NT) cp_async4(dq + i, gq + i);
    }
    float* dg = reinterpret_cast<float*>(smem + O::oGeo) + bf * ET * kGeoStride;
    const float* gg = A.geo + f0 * kGeoStride;
    for (int i = tid; i < n * kGeoStride / 4; i += NT) cp_async16(dg + 4 * i, gg + 4 * i);
    int32_t* dc = reinterpret_cast<int32_t*>(smem + O::oConn) + bf * ET * 4;
    const int32_t* gc = A.conn + f0 * 4;
    for (int i = tid; i < n; i += NT) cp_async16(dc + 4 * i, gc + 4 * i);
    unsigned char* dl = smem + O::oFL + bf * O::kFL;
    const uint8_t* gl = A.face_list + size_t(t) * O::kFL;
    for (int i = tid; i < int(O::kFL / 16); i += NT) cp_async16(dl + 16 * i, gl + 16 * i);
  };
  prefetch(blockIdx.x, 0);
  cp_async_commit();
  if (A.pdl) griddep_wait();         // the closure's increments bD, read by outer faces

  double cled = 0.0;                 // this CTA's ledger sums (threads 0..4)
  int iter = 0;
  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x, ++iter) {
    const int64_t e0 = int64_t(tile) * ET;
    const int nE = int((A.K - e0) < ET ? (A.K - e0) : int64_t(ET));
    const int buf = iter & 1;
    const float* sQ = reinterpret_cast<const float*>(smem + O::oQ) + buf * O::kQT;
    const float* sGeo = reinterpret_cast<const float*>(smem + O::oGeo) + buf * ET * kGeoStride;
    const int32_t* sConn = reinterpret_cast<const int32_t*>(smem + O::oConn) + buf * ET * 4;
    const uint8_t* sFL = smem + O::oFL + buf * O::kFL;      // header, then (le << 2 | f)
    cp_async_wait_all();
    __syncthreads();   // this tile's data is in; the previous tile is finished
    if (*sAbort) break;

    // neighbour traces of faces whose neighbour lies outside the tile, into
    // G (variable v, element le, face node fm)
    // face list groups: [0, aEnd) inside the tile, [aEnd, bEnd) to other
    // tiles, [bEnd, cEnd) outer faces (items = face x face node)
    const int32_t* hdr = reinterpret_cast<const int32_t*>(sFL);
    const int aEnd = hdr[1] * Nfp, bEnd = (hdr[1] + hdr[2]) * Nfp, cEnd = hdr[0] * Nfp;
    const int e0i = int(e0);
    for (int it = aEnd + tid; it < bEnd; it += NT) {
      const int fi = it / Nfp, m = it - (it / Nfp) * Nfp;
      const int ent = sFL[16 + fi], le = ent >> 2, f = ent & 3, fm = f * Nfp + m;
      if (!DG_IN(le < nE, A.status)) continue;
      const int32_t c = sConn[le * 4 + f];
      const int64_t e2 = c >> 5;
      const int f2 = (c >> 3) & 3, o = c & 7;
      if (!DG_IN(c >= 0 && e2 < A.K_all && o < 6, A.status)) continue;
      const int n2 = sTbl[((f * 4 + f2) * 6 + o) * Nfp + m];
      if (!DG_IN(n2 < Np, A.status)) continue;
      const float* src = A.q_in + e2 * 5 * Np + n2;
#pragma unroll
      for (int v = 0; v < 5; ++v) cp_async4(sG + v * kG + le * NF + fm, src + v * Np);
    }
    cp_async_commit();
    prefetch(tile + gridDim.x, buf ^ 1);
    cp_async_commit();

    // ---- volume: reference-direction fluxes into A columns [0, 3 Np). A warp
    // takes 8 elements x 4 nodes, so the 32 stores of one (direction,
    // variable) fall on 32 banks: bank 4 ((5 le + v) mod 8) + (k mod 4)
    for (int wi = warp; wi < O::NB * O::EG; wi += NT / 32) {
      const int nb = wi % O::NB, eg = wi / O::NB;
      const int le = 8 * eg + (lane >> 2), n = 4 * nb + (lane & 3);
      if (le >= nE || n >= Np) continue;
      float q[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = sQ[(le * 5 + v) * Np + n];
      float rinv, u[3], pp;
      prim_tc(q, b, rinv, u, pp);
      if (!(b.rho0 + q[0] > 0.0f) || !(b.p0 + pp > 0.0f) || !isfinite(q[4]) || !isfinite(pp))
        atomicOr(A.status, kStatusBadState);
      const float H = b.H0 + q[4] + pp;
      float F[3][5];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        F[d][0] = q[1 + d];
        F[d][1] = q[1] * u[d];
        F[d][2] = q[2] * u[d];
        F[d][3] = q[3] * u[d];
        F[d][1 + d] += pp;
        F[d][4] = u[d] * H;
      }
      const float* dr = sGeo + le * kGeoStride + kGeoDrdx;
      uint32_t roff[5], coff[3];
#pragma unroll
      for (int v = 0; v < 5; ++v) roff[v] = tc::kmajor_offset(le * 5 + v, 0, SBO);
#pragma unroll
      for (int a = 0; a < 3; ++a) coff[a] = tc::kmajor_offset(0, a * Np + n, SBO);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float m0 = dr[a * 3], m1 = dr[a * 3 + 1], m2 = dr[a * 3 + 2];
#pragma unroll
        for (int v = 0; v < 5; ++v)
          store_a(sAhi, roff[v] + coff[a], m0 * F[0][v] + m1 * F[1][v] + m2 * F[2][v]);
      }
    }
    cp_async_wait_group1();            // the gathers; the next tile may still fly
    __syncthreads();

    // ---- faces: jumps Fscale (n.F(q-) - F*) into A columns [3 Np, 3 Np + 4 Nfp),
    // a face between two elements of the tile once (both jumps: Fscale (A + B)
    // and Fscale' (A - B), A = (n.F(q-) - n.F(q+)) / 2, B = lambda (q+ - q-) / 2)
    float led[5] = {0, 0, 0, 0, 0};
    bool any_bdry = false;
    for (int it = tid; it < cEnd; it += NT) {
      const int fi = it / Nfp, m = it - (it / Nfp) * Nfp;
      const int ent = sFL[16 + fi], le = ent >> 2, f = ent & 3, fm = f * Nfp + m;
      if (!DG_IN(le < nE, A.status)) continue;
      const int n = sFmask[f * Nfp + m];
      if (!DG_IN(n >= 0 && n < Np, A.status)) continue;
      float qm[5], qp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qm[v] = sQ[(le * 5 + v) * Np + n];
      const float* geo = sGeo + le * kGeoStride;
      const float nv[3] = {geo[kGeoNrm + 3 * f], geo[kGeoNrm + 3 * f + 1], geo[kGeoNrm + 3 * f + 2]};
      const int32_t c = sConn[le * 4 + f];
      const float fs = geo[kGeoFscale + f];
      float fnm[5], hA[5], hB[5];
      if (it < aEnd) {
        // both elements in the tile
        const int le2 = (c >> 5) - e0i, f2 = (c >> 3) & 3, o = c & 7;
        if (!DG_IN(c >= 0 && le2 >= 0 && le2 < nE && o < 6, A.status)) continue;
        const int tb = ((f * 4 + f2) * 6 + o) * Nfp + m;
        if (!DG_IN(sTbl[tb] < Np && sTbl[96 * Nfp + tb] < Nfp, A.status)) continue;
        const float* src = sQ + le2 * 5 * Np + sTbl[tb];
#pragma unroll
        for (int v = 0; v < 5; ++v) qp[v] = src[v * Np];
        llf_parts_tc(qm, qp, nv, b, fnm, hA, hB);
        const int fm2 = f2 * Nfp + sTbl[96 * Nfp + tb];
        const float fs2 = sGeo[le2 * kGeoStride + kGeoFscale + f2];
        const uint32_t c1 = tc::kmajor_offset(0, 3 * Np + fm, SBO);
        const uint32_t c2 = tc::kmajor_offset(0, 3 * Np + fm2, SBO);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          store_a(sAhi, tc::kmajor_offset(le * 5 + v, 0, SBO) + c1, fs * (hA[v] + hB[v]));
          store_a(sAhi, tc::kmajor_offset(le2 * 5 + v, 0, SBO) + c2, fs2 * (hA[v] - hB[v]));
        }
      } else if (it < bEnd) {
        // neighbour in another tile: its trace was gathered into G
#pragma unroll
        for (int v = 0; v < 5; ++v) qp[v] = sG[v * kG + le * NF + fm];
        llf_parts_tc(qm, qp, nv, b, fnm, hA, hB);
        const uint32_t c1 = tc::kmajor_offset(0, 3 * Np + fm, SBO);
#pragma unroll
        for (int v = 0; v < 5; ++v)
          store_a(sAhi, tc::kmajor_offset(le * 5 + v, 0, SBO) + c1, fs * (hA[v] + hB[v]));
      } else {
        // outer face: ghost state, and the flux integral for the ledger
        const int mode = A.bc_mode[(-1 - c) & 7];
        if (mode == 3) {
          if (!DG_IN(c < 0 && ((-1 - c) >> 3) < A.nb, A.status)) continue;
          const float D = A.bD ? A.bD[size_t((-1 - c) >> 3) * Nfp + m] : 0.0f;
          ghost_learned_f(qm, nv, bg, D, qp);
        } else {
          ghost_state_f(mode, qm, nv, bg, qp);
        }
        llf_parts_tc(qm, qp, nv, b, fnm, hA, hB);
        const float wsj = sW[fm] * geo[kGeoSJ + f];
        const uint32_t c1 = tc::kmajor_offset(0, 3 * Np + fm, SBO);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          store_a(sAhi, tc::kmajor_offset(le * 5 + v, 0, SBO) + c1, fs * (hA[v] + hB[v]));
          led[v] += wsj * (fnm[v] - hA[v] - hB[v]);     // F* = n.F(q-) - A - B
        }
        any_bdry = true;
      }
    }
    // boundary-flux ledger of this tile
    if (__syncthreads_or(any_bdry)) {
      for (int v = 0; v < 5; ++v) {
        float x = led[v];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) sRed[warp * 5 + v] = double(x);
      }
      __syncthreads();
      if (tid < 5) {
        double acc = 0.0;
        for (int w = 0; w < NT / 32; ++w) acc += sRed[w * 5 + tid];
        cled += acc;
      }
    }
    // every A entry is written: split each 16-byte chunk of the head image
    // into its tf32 head (in place) and tail (same offset in the tail image);
    // the one-pass variant gives the float32 values to the MMA as they are
    if constexpr (S == 2) {
    __syncthreads();
    for (int i = tid; i < int(O::kABytes / 16); i += NT) {
      const float4 x = *reinterpret_cast<const float4*>(sAhi + 16 * i);
      float4 h, l;
      h.x = tc::to_tf32(x.x);
      h.y = tc::to_tf32(x.y);
      h.z = tc::to_tf32(x.z);
      h.w = tc::to_tf32(x.w);
      l.x = tc::to_tf32(x.x - h.x);
      l.y = tc::to_tf32(x.y - h.y);
      l.z = tc::to_tf32(x.z - h.z);
      l.w = tc::to_tf32(x.w - h.w);
      *reinterpret_cast<float4*>(sAhi + 16 * i) = h;
      *reinterpret_cast<float4*>(sAlo + 16 * i) = l;
    }
    }
    // operand writes become visible to the tensor cores
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      // descriptors of k-step s: the start address field (bits 0-13, in
      // 16-byte units) advances by 256 bytes = 16 units per step
      const uint64_t dAhi = tc::smem_desc(tc::smem_addr(sAhi), 128u, SBO);
      const uint64_t dBhi = tc::smem_desc(tc::smem_addr(smem + O::oBhi), 128u, SBO);
      if constexpr (S == 2) {
        const uint64_t dAlo = tc::smem_desc(tc::smem_addr(sAlo), 128u, SBO);
        const uint64_t dBlo = tc::smem_desc(tc::smem_addr(smem + O::oBlo), 128u, SBO);
#pragma unroll
        for (int s = 0; s < K / 8; ++s) {
          const uint64_t step = 16u * uint64_t(s);
          tc::mma_tf32(tmem, dAhi + step, dBhi + step, idesc, s > 0 ? 1u : 0u);
          tc::mma_tf32(tmem, dAhi + step, dBlo + step, idesc, 1u);
          tc::mma_tf32(tmem, dAlo + step, dBhi + step, idesc, 1u);
        }
      } else {
#pragma unroll
        for (int s = 0; s < K / 8; ++s) {
          const uint64_t step = 16u * uint64_t(s);
          tc::mma_tf32(tmem, dAhi + step, dBhi + step, idesc, s > 0 ? 1u : 0u);
        }
      }
      tc::mma_commit(mbar);
    }
    // the residuals the Runge-Kutta pass will read, loaded while the MMAs run
    constexpr int RI = (O::kQT + NT - 1) / NT;
    const int64_t base = e0 * 5 * Np;
    float rres[RI];
#pragma unroll
    for (int s = 0; s < RI; ++s) {
      const int i = tid + s * NT;
      rres[s] = (A.a != 0.0f && i < nE * 5 * Np) ? A.res[base + i] : 0.0f;
    }

    // ---- accumulator rows -> R [row][SO]: warp w (w < 4) holds rows
    // 16 w .. 16 w + 15 in its lanes 0..15
    if (warp < 4) {
      // one lane per warp polls (suspended up to 200 ns per try), the warp
      // follows its verdict
      uint32_t ok = 0;
      if (lane == 0) ok = tc::mbar_wait_hint(mbar, phase, kHintTries, 200u) ? 1u : 0u;
      const bool done = __shfl_sync(0xffffffffu, ok, 0) != 0;
      if (!done) {
        if (lane == 0) {
          atomicOr(A.status, kStatusTimeout);
          *sAbort = 1;
        }
      } else {
        tc::fence_after_sync();
        float d[32];
        tc::tmem_ld_32x32b_x32(tmem + (uint32_t(32 * warp) << 16), d);
        const int row = 16 * warp + lane;
        if (lane < 16 && row < 5 * nE) {
#pragma unroll
          for (int j = 0; j < (Np < 32 ? Np : 32); ++j) sR[row * SO + j] = d[j];
        }
        if constexpr (Np > 32) {
          // columns 32 .. 39 (p = 4: Np = 35)
          float d8[8];
          tc::tmem_ld_32x32b_x8(tmem + (uint32_t(32 * warp) << 16) + 32u, d8);
          if (lane < 16 && row < 5 * nE) {
#pragma unroll
            for (int j = 32; j < Np; ++j) sR[row * SO + j] = d8[j - 32];
          }
        }
      }
    }
    phase ^= 1u;
    tc::fence_before_sync();
    __syncthreads();

    // ---- Runge-Kutta update, coalesced over the tile's state
#pragma unroll
    for (int s = 0; s < RI; ++s) {
      const int i = tid + s * NT;
      if (i < nE * 5 * Np) {
        const int row = i / Np, n = i - (i / Np) * Np;
        const float res = A.a * rres[s] + A.dt * sR[row * SO + n];
        A.res[base + i] = res;
        A.q_out[base + i] = sQ[i] + A.b * res;
      }
    }
  }
  cp_async_wait_all();
  // a wait that gave up may leave MMAs in flight: give them a bounded chance
  // to finish before the tensor memory is released. `phase` was flipped after
  // the wait that gave up, so that wait's parity is phase ^ 1 (waiting on
  // `phase` itself would ask about the phase before it, complete long ago).
  if (*sAbort && tid == 0) tc::mbar_wait(mbar, phase ^ 1u, kWaitTries);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, O::TCOLS);
  }
  ledger_finish(A.led, cled);
}

// orders 1..4 x images 1, 2: f(P, S) for the runtime pair (p, images)
#define DGK_TC_DISPATCH(p, images, F)                            \
  switch ((p) * 4 + (images)) {                                  \
    case 1 * 4 + 1: F(1, 1); case 1 * 4 + 2: F(1, 2);             \
    case 2 * 4 + 1: F(2, 1); case 2 * 4 + 2: F(2, 2);             \
    case 3 * 4 + 1: F(3, 1); case 3 * 4 + 2: F(3, 2);             \
    case 4 * 4 + 1: F(4, 1); default: F(4, 2);                    \
  }

size_t stage_tc_ops_bytes(int p, int images) {
#define F(P, S) return OrderTC<P, S>::kOpsBytes
  DGK_TC_DISPATCH(p, images, F)
#undef F
}

int stage_tc_tile_elems(int) { return 12; }

int stage_tc_ctas_per_sm(int p) { return p <= 3 ? OrderTC<3>::CPS : OrderTC<4>::CPS; }

// Host-side image of B = [-Dr | -Ds | -Dt | LIFT] in the operand layout:
// with S = 2 split into tf32 head and tail, with S = 1 the tf32 rounding
// alone; followed by the face weights.
template <int P, int S>
static void build_ops_impl(const double* Dr, const double* Ds, const double* Dt, const double* LIFT,
                           const double* face_w, unsigned char* out) {
  using O = OrderTC<P, S>;
  auto tf32 = [](float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;   // round to nearest, ties away from zero
    float y;
    std::memcpy(&y, &u, 4);
    return y;
  };
  std::memset(out, 0, O::kOpsBytes);
  float* hi = reinterpret_cast<float*>(out);
  float* lo = reinterpret_cast<float*>(out + O::kBBytes);
  for (int i = 0; i < O::Np; ++i)
    for (int k = 0; k < O::KU; ++k) {
      double v;
      if (k < 3 * O::Np) {
        const double* D = k < O::Np ? Dr : (k < 2 * O::Np ? Ds : Dt);
        v = -D[i * O::Np + (k % O::Np)];
      } else {
        v = LIFT[i * O::NF + (k - 3 * O::Np)];
      }
      const float x = float(v);
      const float h = tf32(x);
      const uint32_t off = tc::kmajor_offset(i, k, O::SBO) / 4;
      hi[off] = h;
      if constexpr (S == 2) lo[off] = tf32(x - h);
    }
  float* w = reinterpret_cast<float*>(out + S * O::kBBytes);
  for (int m = 0; m < O::NF; ++m) w[m] = float(face_w[m]);
}

void build_tc_ops(int p, int images, const double* Dr, const double* Ds, const double* Dt,
                  const double* LIFT, const double* face_w, unsigned char* out) {
#define F(P, S) return build_ops_impl<P, S>(Dr, Ds, Dt, LIFT, face_w, out)
  DGK_TC_DISPATCH(p, images, F)
#undef F
}

template <int P, int S>
static cudaError_t prepare_tc_impl(int* bps) {
  cudaError_t e = cudaFuncSetAttribute(stage_tc_kernel<P, S>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(OrderTC<P, S>::bytes));
  if (e != cudaSuccess) return e;
  // the whole unified L1 as shared memory (two CTAs per SM at p <= 3)
  e = cudaFuncSetAttribute(stage_tc_kernel<P, S>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           int(cudaSharedmemCarveoutMaxShared));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, stage_tc_kernel<P, S>,
                                                       OrderTC<P, S>::NT, OrderTC<P, S>::bytes);
}

cudaError_t stage_tc_prepare(int p, int images, int* bps) {
#define F(P, S) return prepare_tc_impl<P, S>(bps)
  DGK_TC_DISPATCH(p, images, F)
#undef F
}

cudaError_t launch_stage_tc(int p, int images, const StageArgsF32& a, int grid, cudaStream_t s) {
  const bool pdl = a.pdl != 0;
#define F(P, S)                                                                               \
  return launch_stage_kernel(stage_tc_kernel<P, S>, grid, OrderTC<P, S>::NT, OrderTC<P, S>::bytes, \
                             s, a, pdl)
  DGK_TC_DISPATCH(p, images, F)
#undef F
}

#undef DGK_TC_DISPATCH

}  // namespace dgk
