// Float64 Runge-Kutta stage of the nodal DG Euler solver: one fused kernel
// per stage that evaluates the semi-discrete operator f(q) of Eq. 12 on a
// tile of elements and applies the 2N-storage update in the same pass.
//
// Per tile (ET consecutive elements, one CTA, persistent over tiles):
//   1. stage the tile's state, geometry and face connections in shared memory
//      (contiguous, coalesced loads);
//   2. volume: at every node the Euler fluxes F, G, H (Eq. 1 with the
//      ideal-gas closure of Eq. 2), folded with the metric into the
//      reference-direction fluxes Fr = rx F + ry G + rz H (and s, t);
//   3. faces: at every face node the own trace, the neighbour's trace
//      (gathered through the face connection and the orientation table) or a
//      ghost state on outer faces, the local Lax-Friedrichs flux F* and the
//      jump Fscale (n.F(q-) - F*); outer faces also add their F* integral to
//      the tile's boundary-flux ledger (fixed-order, no atomics);
//   4. per node: rhs = -(Dr Fr + Ds Fs + Dt Ft) + LIFT dF, then
//      res <- a res + dt rhs; q_out <- q + b res.
// Every face is evaluated once from each side; the two sides form F* from
// the same pair of states, so no face buffer or atomic is needed.
// The float64 pipe bounds this kernel on GB300; the operators therefore live
// in shared memory, transposed so that the lanes of a warp (consecutive
// nodes) read consecutive words.
#include <cmath>

#include "dg_device.cuh"
#include "dg_physics.cuh"

namespace dgk {

template <int P>
struct Order {
  static constexpr int Np = (P + 1) * (P + 2) * (P + 3) / 6;
  static constexpr int Nfp = (P + 1) * (P + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  // elements per tile; one thread per (element, node), rounded up to whole warps
  static constexpr int ET = P == 1 ? 64 : P == 2 ? 24 : P == 3 ? 12 : 8;
  static constexpr int NT = (ET * Np + 31) / 32 * 32;
  static constexpr int kOps = 3 * Np * Np + NF * Np + NF;
  static constexpr int kTbl = 4 * 4 * 6 * Nfp;
  // shared memory (in doubles unless noted)
  static constexpr int oOps = 0;
  static constexpr int oQ = oOps + kOps;
  static constexpr int oF = oQ + ET * 5 * Np;
  static constexpr int oDF = oF + ET * 15 * Np;
  static constexpr int oGeo = oDF + ET * 5 * NF;
  static constexpr int oRed = oGeo + ET * kGeoStride;
  static constexpr int nWarps = (NT + 31) / 32;
  static constexpr int oEnd = oRed + nWarps * 5;
  // integer region after the doubles
  static constexpr size_t bytes_double = size_t(oEnd) * 8;
  static constexpr size_t oConnB = bytes_double;                       // ET*4 int32
  static constexpr size_t oFmaskB = oConnB + size_t(ET) * 4 * 4;       // 4*Nfp int32
  static constexpr size_t oTblB = oFmaskB + size_t(4) * Nfp * 4;       // 2 kTbl bytes
  static constexpr size_t kFL = 16 + (4 * size_t(ET) + 15) / 16 * 16;   // face list row
  static constexpr size_t oFLB = (oTblB + 2 * kTbl + 15) / 16 * 16;
  static constexpr size_t bytes = (oFLB + kFL + 15) / 16 * 16;
};

template <int P>
__global__ void __launch_bounds__(Order<P>::NT)
stage_fp64_kernel(const StageArgs A) {
  using O = Order<P>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF, ET = O::ET, NT = O::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* sOps = sm + O::oOps;
  double* sQ = sm + O::oQ;
  double* sF = sm + O::oF;
  double* sDF = sm + O::oDF;
  double* sGeo = sm + O::oGeo;
  double* sRed = sm + O::oRed;
  int32_t* sConn = reinterpret_cast<int32_t*>(smem_raw + O::oConnB);
  int32_t* sFmask = reinterpret_cast<int32_t*>(smem_raw + O::oFmaskB);
  uint8_t* sTbl = smem_raw + O::oTblB;
  const double* DrT = sOps;
  const double* DsT = sOps + Np * Np;
  const double* DtT = sOps + 2 * Np * Np;
  const double* LiftT = sOps + 3 * Np * Np;
  const double* faceW = LiftT + NF * Np;
  const int tid = threadIdx.x;

  for (int i = tid; i < O::kOps; i += NT) sOps[i] = A.ops[i];
  for (int i = tid; i < 2 * O::kTbl; i += NT) sTbl[i] = A.nbr_tbl[i];   // volume- and face-node tables
  uint8_t* sFL = smem_raw + O::oFLB;
  for (int i = tid; i < 4 * Nfp; i += NT) sFmask[i] = A.fmask[i];
  const Gas g = A.gas;

  double cled = 0.0;                 // this CTA's ledger sums (threads 0..4)
  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
    const int64_t e0 = int64_t(tile) * ET;
    const int nE = int((A.K - e0) < ET ? (A.K - e0) : int64_t(ET));
    __syncthreads();  // previous tile finished with the shared buffers
    {
      const double* gq = A.q_in + e0 * 5 * Np;
      for (int i = tid; i < nE * 5 * Np; i += NT) sQ[i] = gq[i];
      const double* gg = A.geo + e0 * kGeoStride;
      for (int i = tid; i < nE * kGeoStride; i += NT) sGeo[i] = gg[i];
      const int32_t* gc = A.conn + e0 * 4;
      for (int i = tid; i < nE * 4; i += NT) sConn[i] = gc[i];
      const uint8_t* gl = A.face_list + size_t(tile) * O::kFL;
      for (int i = tid; i < int(O::kFL); i += NT) sFL[i] = gl[i];
    }
    __syncthreads();

    // ---- volume fluxes at nodes
    {
      const int le = tid / Np, n = tid - (tid / Np) * Np;
      if (le < nE) {
        double q[5];
        for (int v = 0; v < 5; ++v) q[v] = sQ[(le * 5 + v) * Np + n];
        double rinv, u[3], p;
        pressure_and_velocity(q, g.gm1, rinv, u, p);
        if (!(q[0] > 0.0) || !(p > 0.0) || !isfinite(q[4]) || !isfinite(p))
          atomicOr(A.status, kStatusBadState);
        double F[3][5];
        for (int d = 0; d < 3; ++d) {
          F[d][0] = q[1 + d];
          F[d][1] = q[1] * u[d];
          F[d][2] = q[2] * u[d];
          F[d][3] = q[3] * u[d];
          F[d][1 + d] += p;
          F[d][4] = u[d] * (q[4] + p);
        }
        const double* dr = sGeo + le * kGeoStride + kGeoDrdx;
        for (int a = 0; a < 3; ++a) {
          const double m0 = dr[a * 3], m1 = dr[a * 3 + 1], m2 = dr[a * 3 + 2];
          for (int v = 0; v < 5; ++v)
            sF[(le * 15 + a * 5 + v) * Np + n] = m0 * F[0][v] + m1 * F[1][v] + m2 * F[2][v];
        }
      }
    }

    // ---- face fluxes at the nodes of the tile's listed faces. A face between
    // two elements of the tile is listed once, under its lower element, which
    // writes both jumps: with A = (n.F(q-) - n.F(q+)) / 2 and
    // B = lambda (q+ - q-) / 2, Fscale (A + B) for itself and Fscale' (A - B)
    // for the neighbour (normal -n, traces swapped).
    double led[5] = {0, 0, 0, 0, 0};
    bool any_bdry = false;
    const int nF = *reinterpret_cast<const int32_t*>(sFL);
    for (int it = tid; it < nF * Nfp; it += NT) {
      const int fi = it / Nfp, m = it - (it / Nfp) * Nfp;
      const int ent = sFL[16 + fi], le = ent >> 2, f = ent & 3, fm = f * Nfp + m;
      if (!DG_IN(le < nE, A.status)) continue;
      const int n = sFmask[f * Nfp + m];
      if (!DG_IN(n >= 0 && n < Np, A.status)) continue;
      double qm[5], qp[5];
      for (int v = 0; v < 5; ++v) qm[v] = sQ[(le * 5 + v) * Np + n];
      const double* geo = sGeo + le * kGeoStride;
      const double nv[3] = {geo[kGeoNrm + 3 * f], geo[kGeoNrm + 3 * f + 1], geo[kGeoNrm + 3 * f + 2]};
      const int32_t c = sConn[le * 4 + f];
      const int le2 = (c >= 0) ? int((c >> 5) - e0) : -1;
      const bool inside = c >= 0 && le2 >= 0 && le2 < nE;   // then le2 > le (face list)
      int f2 = 0, m2 = 0;
      if (inside) {
        f2 = (c >> 3) & 3;
        const int o = c & 7;
        if (!DG_IN(o < 6, A.status)) continue;
        const int n2 = sTbl[((f * 4 + f2) * 6 + o) * Nfp + m];
        m2 = sTbl[O::kTbl + ((f * 4 + f2) * 6 + o) * Nfp + m];
        if (!DG_IN(n2 < Np && m2 < Nfp, A.status)) continue;
        for (int v = 0; v < 5; ++v) qp[v] = sQ[(le2 * 5 + v) * Np + n2];
      } else if (c >= 0) {
        const int64_t e2 = c >> 5;
        const int f2 = (c >> 3) & 3, o = c & 7;
        if (!DG_IN(e2 < A.K_all && o < 6, A.status)) continue;
        const int n2 = sTbl[((f * 4 + f2) * 6 + o) * Nfp + m];
        if (!DG_IN(n2 < Np, A.status)) continue;
        const double* src = A.q_in + e2 * 5 * Np + n2;
        for (int v = 0; v < 5; ++v) qp[v] = __ldg(src + v * Np);
      } else {
        ghost_state(A.bc_mode[(-1 - c) & 7], qm, nv, g, A.inflow, qp);
      }
      double fnm[5], fnp[5], lm, lp;
      normal_flux(qm, nv, g, fnm, lm);
      normal_flux(qp, nv, g, fnp, lp);
      const double lam = fmax(lm, lp);
      const double fs = geo[kGeoFscale + f];
      const double fs2 = inside ? sGeo[le2 * kGeoStride + kGeoFscale + f2] : 0.0;
      for (int v = 0; v < 5; ++v) {
        const double hA = 0.5 * (fnm[v] - fnp[v]), hB = 0.5 * lam * (qp[v] - qm[v]);
        sDF[(le * 5 + v) * NF + fm] = fs * (hA + hB);
        if (inside) sDF[(le2 * 5 + v) * NF + f2 * Nfp + m2] = fs2 * (hA - hB);
        if (c < 0) led[v] += faceW[fm] * geo[kGeoSJ + f] * (0.5 * (fnm[v] + fnp[v]) - hB);
      }
      any_bdry |= (c < 0);
    }
    // boundary-flux ledger of this tile: fixed-order block reduction
    if (__syncthreads_or(any_bdry)) {
      const int lane = tid & 31, warp = tid >> 5;
      for (int v = 0; v < 5; ++v) {
        double x = led[v];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) sRed[warp * 5 + v] = x;
      }
      __syncthreads();
      if (tid < 5) {
        double acc = 0.0;
        for (int w = 0; w < O::nWarps; ++w) acc += sRed[w * 5 + tid];
        cled += acc;
      }
    }
    __syncthreads();

    // ---- per node: contraction, lift, Runge-Kutta update
    {
      const int le = tid / Np, n = tid - (tid / Np) * Np;
      if (le < nE) {
        double acc[5] = {0, 0, 0, 0, 0};
        const double* Fr = sF + (le * 15) * Np;
        const double* Fs = Fr + 5 * Np;
        const double* Ft = Fr + 10 * Np;
#pragma unroll 4
        for (int j = 0; j < Np; ++j) {
          const double dr = DrT[j * Np + n], ds = DsT[j * Np + n], dt = DtT[j * Np + n];
#pragma unroll
          for (int v = 0; v < 5; ++v)
            acc[v] += dr * Fr[v * Np + j] + ds * Fs[v * Np + j] + dt * Ft[v * Np + j];
        }
        double out[5];
        for (int v = 0; v < 5; ++v) out[v] = -acc[v];
        const double* dF = sDF + (le * 5) * NF;
#pragma unroll 4
        for (int m = 0; m < NF; ++m) {
          const double l = LiftT[m * Np + n];
#pragma unroll
          for (int v = 0; v < 5; ++v) out[v] += l * dF[v * NF + m];
        }
        const int64_t base = (e0 + le) * 5 * Np + n;
        for (int v = 0; v < 5; ++v) {
          const int64_t ix = base + int64_t(v) * Np;
          const double r = (A.a != 0.0) ? A.a * A.res[ix] + A.dt * out[v] : A.dt * out[v];
          A.res[ix] = r;
          A.q_out[ix] = sQ[(le * 5 + v) * Np + n] + A.b * r;
        }
      }
    }
  }
  ledger_finish(A.led, cled);
}

int stage_tile_elems(int p) {
  switch (p) {
    case 1: return Order<1>::ET;
    case 2: return Order<2>::ET;
    case 3: return Order<3>::ET;
    default: return Order<4>::ET;
  }
}

size_t stage_smem_bytes(int p) {
  switch (p) {
    case 1: return Order<1>::bytes;
    case 2: return Order<2>::bytes;
    case 3: return Order<3>::bytes;
    default: return Order<4>::bytes;
  }
}

template <int P>
static cudaError_t prepare_impl(int* bps) {
  cudaError_t e = cudaFuncSetAttribute(stage_fp64_kernel<P>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(Order<P>::bytes));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, stage_fp64_kernel<P>, Order<P>::NT,
                                                       Order<P>::bytes);
}

cudaError_t stage_prepare(int p, int* bps) {
  switch (p) {
    case 1: return prepare_impl<1>(bps);
    case 2: return prepare_impl<2>(bps);
    case 3: return prepare_impl<3>(bps);
    default: return prepare_impl<4>(bps);
  }
}

cudaError_t launch_stage(int p, const StageArgs& a, int grid, cudaStream_t s) {
  switch (p) {
    case 1: stage_fp64_kernel<1><<<grid, Order<1>::NT, Order<1>::bytes, s>>>(a); break;
    case 2: stage_fp64_kernel<2><<<grid, Order<2>::NT, Order<2>::bytes, s>>>(a); break;
    case 3: stage_fp64_kernel<3><<<grid, Order<3>::NT, Order<3>::bytes, s>>>(a); break;
    default: stage_fp64_kernel<4><<<grid, Order<4>::NT, Order<4>::bytes, s>>>(a); break;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------- small kernels

// Sensor values: out[probe][v] = sum_n row[probe][n] q[elem][v][n]
__global__ void probe_kernel(const double* q, int Np, int n, const int32_t* elem,
                             const double* rows, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * 5) return;
  const int pidx = i / 5, v = i - (i / 5) * 5;
  const double* src = q + (int64_t(elem[pidx]) * 5 + v) * Np;
  const double* row = rows + size_t(pidx) * Np;
  double acc = 0.0;
  for (int j = 0; j < Np; ++j) acc += row[j] * src[j];
  out[i] = acc;
}

cudaError_t launch_probe_sample(const double* q, int Np, int n, const int32_t* elem,
                                const double* rows, double* out, cudaStream_t s) {
  const int threads = 128, blocks = (n * 5 + threads - 1) / threads;
  probe_kernel<<<blocks, threads, 0, s>>>(q, Np, n, elem, rows, out);
  return cudaGetLastError();
}

// Conserved totals: per-block partial sums over a fixed element range, then
// one block adds the partials in order.
__global__ void totals_partial_kernel(const double* q, const double* geo, const double* mw,
                                      int64_t K, int Np, double* partial) {
  __shared__ double red[256 * 5];
  const int tid = threadIdx.x;
  const int64_t per = (K + gridDim.x - 1) / gridDim.x;
  const int64_t lo = per * blockIdx.x, hi = min(K, lo + per);
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t e = lo + tid; e < hi; e += blockDim.x) {
    const double J = geo[e * kGeoStride + kGeoJ];
    for (int v = 0; v < 5; ++v) {
      double s = 0.0;
      for (int j = 0; j < Np; ++j) s += mw[j] * q[(e * 5 + v) * Np + j];
      acc[v] += J * s;
    }
  }
  for (int v = 0; v < 5; ++v) red[tid * 5 + v] = acc[v];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int v = 0; v < 5; ++v) red[tid * 5 + v] += red[(tid + w) * 5 + v];
    __syncthreads();
  }
  if (tid < 5) partial[blockIdx.x * 5 + tid] = red[tid];
}

__global__ void totals_final_kernel(const double* partial, int nblocks, double* out) {
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int i = 0; i < nblocks; ++i) s += partial[i * 5 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

cudaError_t launch_totals(const double* q, const double* geo, const double* mass_w, int64_t K,
                          int Np, double* partial, int nblocks, double* out, cudaStream_t s) {
  totals_partial_kernel<<<nblocks, 256, 0, s>>>(q, geo, mass_w, K, Np, partial);
  totals_final_kernel<<<1, 32, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

}  // namespace dgk
