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
// float64 kernel: one launch per stage, every face evaluated from both
// sides, no atomics; GB300's float64 pipe is left idle except for the
// per-tile boundary-flux sums. The Dr/Ds/Dt contraction and the lift, three
// quarters of the arithmetic, are one product per (variable, element) row
// with the operator columns broadcast from shared memory (see OrderF).
#include <cmath>
#include <cstdint>

#include "cp_async.cuh"
#include "dg_device.cuh"
#include "ghost_f32.cuh"

namespace dgk {

struct BaseF {
  float rho0, p0, gamma, gm1, H0;
};

// velocity, pressure perturbation and 1/rho of a perturbation state
__device__ __forceinline__ void prim_f(const float q[5], const BaseF& b, float& rinv, float u[3],
                                       float& pp) {
  rinv = __fdividef(1.0f, b.rho0 + q[0]);          // 2 ulp: far below the form's tolerance
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
  const float c2 = b.gamma * (b.p0 + pp) * rinv;
  lam = fabsf(un) + (c2 > 0.0f ? c2 * rsqrtf(c2) : 0.0f);
}

// Parts of the LLF flux at a face node: n.F(q-), A = (n.F(q-) - n.F(q+)) / 2,
// B = lambda (q+ - q-) / 2; F* = n.F(q-) - A - B, the jump n.F(q-) - F* = A + B.
__device__ __forceinline__ void llf_parts_f(const float qm[5], const float qp[5], const float n[3],
                                            const BaseF& b, float fnm[5], float hA[5], float hB[5]) {
  float fnp[5], lm, lp;
  normal_flux_f(qm, n, b, fnm, lm);
  normal_flux_f(qp, n, b, fnp, lp);
  const float lam = fmaxf(lm, lp);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    hA[v] = 0.5f * (fnm[v] - fnp[v]);
    hB[v] = 0.5f * lam * (qp[v] - qm[v]);
  }
}

// acc += a * b on two packed float32 lanes (one instruction for two FMAs)
__device__ __forceinline__ void fma2(uint64_t& acc, uint64_t a, uint64_t b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

// Tile of ET = 32 elements. The node and face phases map threads to
// (element, node) and (element, face node) items and write one row per
// (variable, element) of
//   X = [F_r (Np) | F_s (Np) | F_t (Np) | Fscale (n.F - F*) (NF)],
// F_a the metric-folded fluxes; the stage's right-hand side is then the
// product of X with OT = [-Dr | -Ds | -Dt | LIFT]^T (K = 3 Np + NF rows),
// staged in shared memory with its Np columns split into NQ parts of NPQ,
// each padded to NPQ4 (16-byte aligned). In the product a warp owns one
// K part (of NK) and one output part, lane = element: per k it loads the
// five X rows of its element (consecutive lanes read rows of odd stride,
// no bank conflicts) and the part's OT entries once (warp-uniform 16-byte
// broadcasts), which feed 5 x NPQ FMAs in packed float32x2 accumulators.
// The NK partial sums, stored [part][v][n][ET+1] (conflict-free both ways),
// meet in the Runge-Kutta pass.
template <int P>
struct OrderF {
  static constexpr int Np = (P + 1) * (P + 2) * (P + 3) / 6;
  static constexpr int Nfp = (P + 1) * (P + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int ET = 32;
  static constexpr int NQ = P == 4 ? 4 : 2;                 // output parts
  static constexpr int NK = 5;                              // K parts
  static constexpr int NT = 32 * NQ * NK;
  static constexpr int K = 3 * Np + NF;
  static constexpr int KP = (K + NK - 1) / NK;
  static constexpr int NPQ = (Np + NQ - 1) / NQ;
  static constexpr int NPQ2 = (NPQ + 1) / 2 * 2;
  static constexpr int NPQ4 = (NPQ + 3) / 4 * 4;
  static constexpr int OTW = NQ * NPQ4;
  static constexpr int kPart = 5 * Np * (ET + 1);           // floats of one K part's sums
  static constexpr int SXmin = (NK * kPart + 5 * ET - 1) / (5 * ET);
  static constexpr int SX0 = K > SXmin ? K : SXmin;
  static constexpr int SX = SX0 % 2 ? SX0 : SX0 + 1;        // odd row stride of X
  static_assert(NK * kPart <= 5 * ET * SX, "partial sums fit in the X rows");
  static constexpr int kTbl = 4 * 4 * 6 * Nfp;
  static constexpr int minBlocks = P == 4 ? 1 : 2;          // CTAs per SM
  // shared memory, in floats: OT [K][OTW], two buffers of the state
  // [le][v][n] (global layout), X [v*ET + le][SX] (after the product: the
  // partial sums), two buffers of geometry records, face weights. The second
  // state / geometry / connection buffer receives the next tile while this
  // one is computed.
  static constexpr int kQT = ET * 5 * Np;
  static constexpr int oOT = 0;
  static constexpr int oQ = oOT + K * OTW;
  static constexpr int oX = oQ + 2 * kQT;
  static constexpr int oGeo = oX + 5 * ET * SX;
  static constexpr int oW = oGeo + 2 * ET * kGeoStride;
  static constexpr int oEnd = oW + NF;
  static constexpr int nWarps = NT / 32;
  static constexpr size_t oRedB = (size_t(oEnd) * 4 + 15) / 16 * 16;
  static constexpr size_t oConnB = oRedB + size_t(nWarps) * 5 * 8;
  static constexpr size_t kFL = 16 + (4 * size_t(ET) + 15) / 16 * 16;   // face list row (16-byte multiple)
  static_assert(kFL % 16 == 0, "face-list rows are copied in 16-byte pieces");
  static constexpr size_t oFLB = oConnB + 2 * size_t(ET) * 4 * 4;   // two face-list buffers
  static constexpr size_t oFmaskB = oFLB + 2 * kFL;
  static constexpr size_t oTblB = oFmaskB + size_t(4) * Nfp * 4;
  static constexpr size_t bytes = (oTblB + 2 * kTbl + 15) / 16 * 16;
};

template <int P>
__global__ void __launch_bounds__(OrderF<P>::NT, OrderF<P>::minBlocks)
stage_f32_kernel(const StageArgsF32 A) {
  using O = OrderF<P>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF, ET = O::ET, NT = O::NT;
  constexpr int K = O::K, SX = O::SX, NPQ = O::NPQ, NPQ2 = O::NPQ2, NPQ4 = O::NPQ4, OTW = O::OTW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  float* sOT = sm + O::oOT;
  float* sX = sm + O::oX;
  float* faceW = sm + O::oW;
  double* sRed = reinterpret_cast<double*>(smem_raw + O::oRedB);
  int32_t* sFmask = reinterpret_cast<int32_t*>(smem_raw + O::oFmaskB);
  uint8_t* sTbl = smem_raw + O::oTblB;
  const int tid = threadIdx.x;

  // OT from the transposed operators in A.ops ([DrT | DsT | DtT] [j][n] and
  // LiftT [m][n]), volume rows negated; then the face weights
  for (int i = tid; i < K * OTW; i += NT) {
    const int k = i / OTW, c = i - (i / OTW) * OTW;
    const int q = c / NPQ4, j = c - (c / NPQ4) * NPQ4, n = q * NPQ + j;
    float v = 0.0f;
    if (j < NPQ && n < Np)
      v = (k < 3 * Np) ? -A.ops[k * Np + n] : A.ops[3 * Np * Np + (k - 3 * Np) * Np + n];
    sOT[i] = v;
  }
  for (int i = tid; i < NF; i += NT) faceW[i] = A.ops[3 * Np * Np + NF * Np + i];
  for (int i = tid; i < 2 * O::kTbl; i += NT) sTbl[i] = A.nbr_tbl[i];   // volume-node and face-node tables
  for (int i = tid; i < 4 * Nfp; i += NT) sFmask[i] = A.fmask[i];
  const BaseF b{float(A.gas.rho0), float(A.gas.p0), float(A.gas.gamma), float(A.gas.gm1),
                float(A.gas.E0 + A.gas.p0)};
  const BaseGhost bg{float(A.gas.rho0), float(A.gas.p0), float(A.gas.gamma), float(A.gas.gm1),
                     float(A.gas.c0), A.inflow[0], A.inflow[1], A.inflow[2]};

  // asynchronous copy of tile t's state, geometry and connections into buffer bf
  auto prefetch = [&](int t, int bf) {
    if (t >= A.ntiles) return;
    const int64_t f0 = int64_t(t) * ET;
    const int n = int((A.K - f0) < ET ? (A.K - f0) : int64_t(ET));
    float* dq = sm + O::oQ + bf * O::kQT;
    const float* gq = A.q_in + f0 * 5 * Np;
    if constexpr ((5 * Np) % 4 == 0) {              // 16-byte rows of the state
      for (int i = tid; i < n * 5 * Np / 4; i += NT) cp_async16(dq + 4 * i, gq + 4 * i);
    } else {
      for (int i = tid; i < n * 5 * Np; i += NT) cp_async4(dq + i, gq + i);
    }
    float* dg = sm + O::oGeo + bf * ET * kGeoStride;
    const float* gg = A.geo + f0 * kGeoStride;
    for (int i = tid; i < n * kGeoStride / 4; i += NT) cp_async16(dg + 4 * i, gg + 4 * i);
    int32_t* dc = reinterpret_cast<int32_t*>(smem_raw + O::oConnB) + bf * ET * 4;
    const int32_t* gc = A.conn + f0 * 4;
    for (int i = tid; i < n; i += NT) cp_async16(dc + 4 * i, gc + 4 * i);
    unsigned char* dl = smem_raw + O::oFLB + bf * O::kFL;
    const uint8_t* gl = A.face_list + size_t(t) * O::kFL;
    for (int i = tid; i < int(O::kFL / 16); i += NT) cp_async16(dl + 16 * i, gl + 16 * i);
  };
  prefetch(blockIdx.x, 0);
  cp_async_commit();
  if (A.pdl) griddep_wait();         // the closure's increments bD, read by outer faces

  int iter = 0;
  double cled = 0.0;                 // this CTA's ledger sums (threads 0..4)
  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x, ++iter) {
    const int64_t e0 = int64_t(tile) * ET;
    const int e0i = int(e0);
    const int nE = int((A.K - e0) < ET ? (A.K - e0) : int64_t(ET));
    const int buf = iter & 1;
    const float* sQ = sm + O::oQ + buf * O::kQT;
    const float* sGeo = sm + O::oGeo + buf * ET * kGeoStride;
    const int32_t* sConn = reinterpret_cast<const int32_t*>(smem_raw + O::oConnB) + buf * ET * 4;
    const uint8_t* sFL = smem_raw + O::oFLB + buf * O::kFL;   // count, then (le << 2 | f)
    cp_async_wait_all();
    __syncthreads();   // this tile's data is in; the previous tile is finished

    // ---- neighbour traces of face nodes whose neighbour lies outside the
    // tile, copied asynchronously into the face columns of X (row v, element
    // le, column 3 Np + fm), where the face phase reads them and then writes
    // the jump; the copies fly while the node phase computes
    // face list groups: [0, aEnd) inside the tile, [aEnd, bEnd) to other
    // tiles, [bEnd, cEnd) outer faces (items = face x face node)
    const int32_t* hdr = reinterpret_cast<const int32_t*>(sFL);
    const int aEnd = hdr[1] * Nfp, bEnd = (hdr[1] + hdr[2]) * Nfp, cEnd = hdr[0] * Nfp;
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
      for (int v = 0; v < 5; ++v) cp_async4(sX + (v * ET + le) * SX + 3 * Np + fm, src + v * Np);
    }
    cp_async_commit();
    prefetch(tile + gridDim.x, buf ^ 1);
    cp_async_commit();

    // ---- volume fluxes (perturbation form) at nodes, folded with the metric
    // two items per trip (two nodes per thread for a full tile): independent
    // load and flux chains side by side
#pragma unroll 2
    for (int it = tid; it < nE * Np; it += NT) {
      const int le = it / Np, n = it - (it / Np) * Np;
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
          sX[(v * ET + le) * SX + a * Np + n] = m0 * F[0][v] + m1 * F[1][v] + m2 * F[2][v];
      }
    }

    cp_async_wait_group1();            // the gathers; the next tile may still fly
    __syncthreads();

    // ---- face fluxes at the nodes of the tile's listed faces. A face between
    // two elements of the tile is listed once, under its lower element, which
    // writes both jumps: with A = (n.F(q-) - n.F(q+)) / 2 and
    // B = lambda (q+ - q-) / 2 the own jump is Fscale (A + B) and the
    // neighbour's (normal -n, traces swapped) Fscale' (A - B). The three
    // groups of the list take their own branch, uniform within almost every
    // warp: no work of one kind runs predicated off in another.
    float led[5] = {0, 0, 0, 0, 0};   // float32 within the tile, float64 across tiles
    bool any_bdry = false;
    for (int it = tid; it < cEnd; it += NT) {
      const int fi = it / Nfp, m = it - (it / Nfp) * Nfp;
      const int ent = sFL[16 + fi], le = ent >> 2, f = ent & 3, fm = f * Nfp + m;
      if (!DG_IN(le < nE, A.status)) continue;
      const int32_t c = sConn[le * 4 + f];
      const int n = sFmask[f * Nfp + m];
      if (!DG_IN(n >= 0 && n < Np, A.status)) continue;
      float qm[5], qp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qm[v] = sQ[(le * 5 + v) * Np + n];
      const float* geo = sGeo + le * kGeoStride;
      const float nv[3] = {geo[kGeoNrm + 3 * f], geo[kGeoNrm + 3 * f + 1], geo[kGeoNrm + 3 * f + 2]};
      float* xf = sX + le * SX + 3 * Np + fm;        // + v * ET * SX
      const float fs = geo[kGeoFscale + f];
      float fnm[5], hA[5], hB[5];
      if (it < aEnd) {
        // both elements in the tile
        const int le2 = (c >> 5) - e0i, f2 = (c >> 3) & 3, o = c & 7;
        if (!DG_IN(c >= 0 && le2 >= 0 && le2 < nE && o < 6, A.status)) continue;
        const int tb = ((f * 4 + f2) * 6 + o) * Nfp + m;
        if (!DG_IN(sTbl[tb] < Np && sTbl[O::kTbl + tb] < Nfp, A.status)) continue;
        const float* src = sQ + le2 * 5 * Np + sTbl[tb];
#pragma unroll
        for (int v = 0; v < 5; ++v) qp[v] = src[v * Np];
        llf_parts_f(qm, qp, nv, b, fnm, hA, hB);
        float* xf2 = sX + le2 * SX + 3 * Np + f2 * Nfp + sTbl[O::kTbl + tb];
        const float fs2 = sGeo[le2 * kGeoStride + kGeoFscale + f2];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          xf[v * ET * SX] = fs * (hA[v] + hB[v]);
          xf2[v * ET * SX] = fs2 * (hA[v] - hB[v]);
        }
      } else if (it < bEnd) {
        // neighbour in another tile: its trace was gathered into the face columns
#pragma unroll
        for (int v = 0; v < 5; ++v) qp[v] = xf[v * ET * SX];
        llf_parts_f(qm, qp, nv, b, fnm, hA, hB);
#pragma unroll
        for (int v = 0; v < 5; ++v) xf[v * ET * SX] = fs * (hA[v] + hB[v]);
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
        llf_parts_f(qm, qp, nv, b, fnm, hA, hB);
        const float wsj = faceW[fm] * geo[kGeoSJ + f];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          xf[v * ET * SX] = fs * (hA[v] + hB[v]);
          led[v] += wsj * (fnm[v] - hA[v] - hB[v]);     // F* = n.F(q-) - A - B
        }
        any_bdry = true;
      }
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
        cled += acc;
      }
    }
    // (the barrier above published the face columns of X; sRed is written
    // again only after the next tile's barriers)

    // ---- X OT: warp = (K part, output part), lane = element
    {
      const int le = tid & 31, w = tid >> 5;
      const int kq = w % O::NK, h = w / O::NK;
      const int k0 = kq * O::KP, k1 = (kq + 1) * O::KP < K ? (kq + 1) * O::KP : K;
      uint64_t acc[5][NPQ2 / 2];
#pragma unroll
      for (int v = 0; v < 5; ++v)
#pragma unroll
        for (int j = 0; j < NPQ2 / 2; ++j) acc[v][j] = 0;
      if (le < nE) {
        const float* x = sX + le * SX;                // row v at + v * ET * SX
        const float* ot = sOT + h * NPQ4;
        // two k per trip: half the loop overhead, still within 96 registers
        // (four spill)
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
          uint64_t op[NPQ2 / 2];
#pragma unroll
          for (int j = 0; j + 1 < NPQ2 / 2; j += 2) {
            const ulonglong2 o = *reinterpret_cast<const ulonglong2*>(ot + k * OTW + 2 * j);
            op[j] = o.x;
            op[j + 1] = o.y;
          }
          if constexpr ((NPQ2 / 2) % 2)
            op[NPQ2 / 2 - 1] = *reinterpret_cast<const uint64_t*>(ot + k * OTW + NPQ2 - 2);
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            uint64_t xx;
            asm("mov.b64 %0, {%1, %1};" : "=l"(xx) : "f"(x[v * ET * SX + k]));
#pragma unroll
            for (int j = 0; j < NPQ2 / 2; ++j) fma2(acc[v][j], op[j], xx);
          }
        }
      }
      __syncthreads();                 // every thread has read its X rows
      if (le < nE) {
        float* part = sX + kq * O::kPart + le;        // [v][n][ET + 1]
#pragma unroll
        for (int v = 0; v < 5; ++v)
#pragma unroll
          for (int j = 0; j < NPQ; ++j) {
            const int n = h * NPQ + j;
            if (n < Np)
              part[(v * Np + n) * (ET + 1)] =
                  __uint_as_float(uint32_t(j % 2 ? acc[v][j / 2] >> 32 : acc[v][j / 2]));
          }
      }
    }
    __syncthreads();

    // the residuals the Runge-Kutta pass will read, loaded after the product
    // (not held in registers through it; the other CTA on the SM covers the wait)
    constexpr int RI = (ET * 5 * Np + NT - 1) / NT;
    const int64_t base = e0 * 5 * Np;
    float rres[RI];
#pragma unroll
    for (int s = 0; s < RI; ++s) {
      const int i = tid + s * NT;
      rres[s] = (A.a != 0.0f && i < nE * 5 * Np) ? A.res[base + i] : 0.0f;
    }

    // ---- Runge-Kutta update, coalesced over the tile's state; output row
    // r = v Np + n of element le is partial-sum row r
    float* const res_t = A.res + base;
    float* const qout_t = A.q_out + base;
#pragma unroll
    for (int s = 0; s < RI; ++s) {
      const int i = tid + s * NT;
      if (i < nE * 5 * Np) {
        const int le = i / (5 * Np), r = i - le * 5 * Np;
        const float* part = sX + r * (ET + 1) + le;
        float rhs = 0.0f;
#pragma unroll
        for (int kq = 0; kq < O::NK; ++kq) rhs += part[kq * O::kPart];
        const float res = A.a * rres[s] + A.dt * rhs;
        res_t[i] = res;
        qout_t[i] = sQ[i] + A.b * res;
      }
    }
  }
  ledger_finish(A.led, cled);
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
  // the whole unified L1 as shared memory, so that two CTAs fit on an SM
  e = cudaFuncSetAttribute(stage_f32_kernel<P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           int(cudaSharedmemCarveoutMaxShared));
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
  const bool pdl = a.pdl != 0;
  switch (p) {
    case 1: return launch_stage_kernel(stage_f32_kernel<1>, grid, OrderF<1>::NT, OrderF<1>::bytes, s, a, pdl);
    case 2: return launch_stage_kernel(stage_f32_kernel<2>, grid, OrderF<2>::NT, OrderF<2>::bytes, s, a, pdl);
    case 3: return launch_stage_kernel(stage_f32_kernel<3>, grid, OrderF<3>::NT, OrderF<3>::bytes, s, a, pdl);
    default: return launch_stage_kernel(stage_f32_kernel<4>, grid, OrderF<4>::NT, OrderF<4>::bytes, s, a, pdl);
  }
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
