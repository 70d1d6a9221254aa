// Float64 Runge-Kutta stage of the paper's own discretisation (Appendix A):
// the weak form of Eq. 10 in the orthonormal basis of Eq. 11 with a Gauss
// rule of degree 2p for the volume integral and one of degree 2p+1 for the
// surface integrals, the local Lax-Friedrichs flux (section 1.1), and the
// 2N-storage update of the caller's Runge-Kutta scheme (Heun's RK2 in
// dg_step). The state stays in nodal values of the same polynomials; the
// operators (modal_ops.cpp) carry the quadrature and the orthonormal mass
// matrix:
//   du_n/dt = sum_a sum_q Sv_a[n][q] G_a(x_q) - sum_f Fscale_f sum_q Sf_f[n][q] F*_q.
//
// Per tile (ET consecutive elements, one CTA, persistent over tiles):
//   1. the tile's nodal state, geometry and face connections into shared
//      memory; the neighbours' nodal values at the nodes matching each own
//      face node (orientation table) gathered next to them;
//   2. faces: at each of the face's quadrature points, the own and the
//      neighbour's trace (interpolated from the face's nodal values) or a
//      ghost state, the LLF flux F*, stored times Fscale; outer faces add
//      wf sJ F* to the tile's ledger sums. The point set of an interior face
//      is the rule of its lower-numbered element (variant 0), which the
//      other element sees through the orientation code (variant 1 + o);
//   3. volume: at each quadrature point the state, the Euler fluxes and
//      their metric fold G_a = sum_d (dr_a/dx_d) F_d;
//   4. per node: the two weighted sums above, then res <- a res + dt rhs,
//      q_out <- q + b res.
// Operators are read through the read-only cache (a few to ~100 KB).
#include <cmath>

#include "dg_device.cuh"
#include "dg_physics.cuh"

namespace dgk {

template <int P>
struct ModalOrder {
  static constexpr int Np = (P + 1) * (P + 2) * (P + 3) / 6;
  static constexpr int Nfp = (P + 1) * (P + 2) / 2;
  static constexpr int n1 = P + 1;                 // Gauss points per collapsed direction
  static constexpr int Nq = n1 * n1 * n1;          // volume rule, degree 2p
  static constexpr int Nfq = n1 * n1;              // face rule, degree 2p + 1
  static constexpr int ET = P == 1 ? 16 : P == 2 ? 8 : P == 3 ? 4 : 2;
  static constexpr int NT = 256;
  static constexpr int nWarps = NT / 32;
  // operator block (doubles)
  static constexpr int oIq = 0;
  static constexpr int oSv = oIq + Nq * Np;
  static constexpr int oIfn = oSv + 3 * Np * Nq;
  static constexpr int oSf = oIfn + 28 * Nfq * Nfp;
  static constexpr int oWf = oSf + 28 * Np * Nfq;
  static constexpr int kOps = oWf + Nfq;
  // shared memory (doubles, then the int32 connections)
  static constexpr int sU = 0;
  static constexpr int sUp = sU + ET * 5 * Np;
  static constexpr int sFs = sUp + ET * 4 * 5 * Nfp;
  static constexpr int sG = sFs + ET * 4 * 5 * Nfq;
  static constexpr int sGeo = sG + ET * 3 * 5 * Nq;
  static constexpr int sRed = sGeo + ET * kGeoStride;
  static constexpr int sEnd = sRed + nWarps * 5;
  static constexpr size_t oConnB = size_t(sEnd) * 8;
  static constexpr size_t bytes = oConnB + size_t(ET) * 4 * 4;
};

int modal_ops_len(int p) {
  switch (p) {
    case 1: return ModalOrder<1>::kOps;
    case 2: return ModalOrder<2>::kOps;
    case 3: return ModalOrder<3>::kOps;
    default: return ModalOrder<4>::kOps;
  }
}

template <int P>
__global__ void __launch_bounds__(ModalOrder<P>::NT)
stage_modal_kernel(const StageArgs A) {
  using O = ModalOrder<P>;
  constexpr int Np = O::Np, Nfp = O::Nfp, Nq = O::Nq, Nfq = O::Nfq, ET = O::ET, NT = O::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* sU = sm + O::sU;
  double* sUp = sm + O::sUp;
  double* sFs = sm + O::sFs;
  double* sG = sm + O::sG;
  double* sGeo = sm + O::sGeo;
  double* sRed = sm + O::sRed;
  int32_t* sConn = reinterpret_cast<int32_t*>(smem_raw + O::oConnB);
  const double* __restrict__ Iq = A.modal_ops + O::oIq;
  const double* __restrict__ Sv = A.modal_ops + O::oSv;
  const double* __restrict__ Ifn = A.modal_ops + O::oIfn;
  const double* __restrict__ Sf = A.modal_ops + O::oSf;
  const double* __restrict__ wf = A.modal_ops + O::oWf;
  const int tid = threadIdx.x;
  const Gas g = A.gas;

  double cled = 0.0;                 // this CTA's ledger sums (threads 0..4)
  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
    const int64_t e0 = int64_t(tile) * ET;
    const int nE = int((A.K - e0) < ET ? (A.K - e0) : int64_t(ET));
    __syncthreads();  // previous tile finished with the shared buffers
    {
      const double* gq = A.q_in + e0 * 5 * Np;
      for (int i = tid; i < nE * 5 * Np; i += NT) sU[i] = gq[i];
      const double* gg = A.geo + e0 * kGeoStride;
      for (int i = tid; i < nE * kGeoStride; i += NT) sGeo[i] = gg[i];
      const int32_t* gc = A.conn + e0 * 4;
      for (int i = tid; i < nE * 4; i += NT) sConn[i] = gc[i];
    }
    __syncthreads();
    // ---- neighbours' nodal values at the nodes matching the own face nodes
    for (int it = tid; it < nE * 4 * Nfp; it += NT) {
      const int le = it / (4 * Nfp), r = it - le * 4 * Nfp, f = r / Nfp, m = r - f * Nfp;
      const int32_t c = sConn[le * 4 + f];
      if (c < 0) continue;
      const int64_t e2 = c >> 5;
      const int f2 = (c >> 3) & 3, o = c & 7;
      if (!DG_IN(e2 < A.K_all && o < 6, A.status)) continue;
      const int n2 = A.nbr_tbl[((f * 4 + f2) * 6 + o) * Nfp + m];
      if (!DG_IN(n2 < Np, A.status)) continue;
      const double* src = A.q_in + e2 * 5 * Np + n2;
#pragma unroll
      for (int v = 0; v < 5; ++v) sUp[((le * 4 + f) * 5 + v) * Nfp + m] = src[v * Np];
    }
    __syncthreads();

    // ---- faces: F* at the face's quadrature points, times Fscale
    double led[5] = {0, 0, 0, 0, 0};
    bool any_bdry = false;
    for (int it = tid; it < nE * 4 * Nfq; it += NT) {
      const int le = it / (4 * Nfq), r = it - le * 4 * Nfq, f = r / Nfq, q = r - f * Nfq;
      const int32_t c = sConn[le * 4 + f];
      const int var = (c < 0 || e0 + le <= int64_t(c >> 5)) ? 0 : 1 + (c & 7);
      if (!DG_IN(var < 7, A.status)) continue;
      const double* I = Ifn + ((f * 7 + var) * Nfq + q) * Nfp;
      double qm[5] = {0, 0, 0, 0, 0}, qp[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < Nfp; ++m) {
        const double w = __ldg(I + m);
        const int n = __ldg(A.fmask + f * Nfp + m);
        if (!DG_IN(n >= 0 && n < Np, A.status)) continue;
#pragma unroll
        for (int v = 0; v < 5; ++v) qm[v] += w * sU[(le * 5 + v) * Np + n];
        if (c >= 0) {
#pragma unroll
          for (int v = 0; v < 5; ++v) qp[v] += w * sUp[((le * 4 + f) * 5 + v) * Nfp + m];
        }
      }
      const double* geo = sGeo + le * kGeoStride;
      const double nv[3] = {geo[kGeoNrm + 3 * f], geo[kGeoNrm + 3 * f + 1], geo[kGeoNrm + 3 * f + 2]};
      if (c < 0) ghost_state(A.bc_mode[(-1 - c) & 7], qm, nv, g, A.inflow, qp);
      double fnm[5], fnp[5], lm, lp;
      normal_flux(qm, nv, g, fnm, lm);
      normal_flux(qp, nv, g, fnp, lp);
      const double lam = fmax(lm, lp);
      const double fs = geo[kGeoFscale + f];
      const double wq = c < 0 ? __ldg(wf + q) * geo[kGeoSJ + f] : 0.0;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double fstar = 0.5 * (fnm[v] + fnp[v]) - 0.5 * lam * (qp[v] - qm[v]);
        sFs[((le * 4 + f) * 5 + v) * Nfq + q] = fs * fstar;
        led[v] += wq * fstar;
      }
      any_bdry |= (c < 0);
    }

    // ---- volume: fluxes at the quadrature points, folded with the metric
    for (int it = tid; it < nE * Nq; it += NT) {
      const int le = it / Nq, q = it - le * Nq;
      double u[5] = {0, 0, 0, 0, 0};
      for (int n = 0; n < Np; ++n) {
        const double w = __ldg(Iq + q * Np + n);
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] += w * sU[(le * 5 + v) * Np + n];
      }
      double rinv, vel[3], p;
      pressure_and_velocity(u, g.gm1, rinv, vel, p);
      if (!(u[0] > 0.0) || !(p > 0.0) || !isfinite(u[4]) || !isfinite(p))
        atomicOr(A.status, kStatusBadState);
      double F[3][5];
      for (int d = 0; d < 3; ++d) {
        F[d][0] = u[1 + d];
        F[d][1] = u[1] * vel[d];
        F[d][2] = u[2] * vel[d];
        F[d][3] = u[3] * vel[d];
        F[d][1 + d] += p;
        F[d][4] = vel[d] * (u[4] + p);
      }
      const double* dr = sGeo + le * kGeoStride + kGeoDrdx;
      for (int a = 0; a < 3; ++a) {
        const double m0 = dr[a * 3], m1 = dr[a * 3 + 1], m2 = dr[a * 3 + 2];
#pragma unroll
        for (int v = 0; v < 5; ++v)
          sG[((le * 3 + a) * 5 + v) * Nq + q] = m0 * F[0][v] + m1 * F[1][v] + m2 * F[2][v];
      }
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

    // ---- per node: weak-form sums and the Runge-Kutta update
    for (int it = tid; it < nE * 5 * Np; it += NT) {
      const int le = it / (5 * Np), r = it - le * 5 * Np, v = r / Np, n = r - v * Np;
      double acc = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double* S = Sv + (a * Np + n) * Nq;
        const double* G = sG + ((le * 3 + a) * 5 + v) * Nq;
        for (int q = 0; q < Nq; ++q) acc += __ldg(S + q) * G[q];
      }
      for (int f = 0; f < 4; ++f) {
        const int32_t c = sConn[le * 4 + f];
        const int var = (c < 0 || e0 + le <= int64_t(c >> 5)) ? 0 : 1 + (c & 7);
        if (!DG_IN(var < 7, A.status)) continue;
        const double* S = Sf + ((f * 7 + var) * Np + n) * Nfq;
        const double* Fs = sFs + ((le * 4 + f) * 5 + v) * Nfq;
        for (int q = 0; q < Nfq; ++q) acc -= __ldg(S + q) * Fs[q];
      }
      const int64_t ix = e0 * 5 * Np + it;
      const double rr = (A.a != 0.0) ? A.a * A.res[ix] + A.dt * acc : A.dt * acc;
      A.res[ix] = rr;
      A.q_out[ix] = sU[it] + A.b * rr;
    }
  }
  ledger_finish(A.led, cled);
}

int stage_modal_tile_elems(int p) {
  switch (p) {
    case 1: return ModalOrder<1>::ET;
    case 2: return ModalOrder<2>::ET;
    case 3: return ModalOrder<3>::ET;
    default: return ModalOrder<4>::ET;
  }
}

template <int P>
static cudaError_t prepare_modal_impl(int* bps) {
  cudaError_t e = cudaFuncSetAttribute(stage_modal_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(ModalOrder<P>::bytes));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, stage_modal_kernel<P>, ModalOrder<P>::NT,
                                                       ModalOrder<P>::bytes);
}

cudaError_t stage_modal_prepare(int p, int* bps) {
  switch (p) {
    case 1: return prepare_modal_impl<1>(bps);
    case 2: return prepare_modal_impl<2>(bps);
    case 3: return prepare_modal_impl<3>(bps);
    default: return prepare_modal_impl<4>(bps);
  }
}

cudaError_t launch_stage_modal(int p, const StageArgs& a, int grid, cudaStream_t s) {
  switch (p) {
    case 1: stage_modal_kernel<1><<<grid, ModalOrder<1>::NT, ModalOrder<1>::bytes, s>>>(a); break;
    case 2: stage_modal_kernel<2><<<grid, ModalOrder<2>::NT, ModalOrder<2>::bytes, s>>>(a); break;
    case 3: stage_modal_kernel<3><<<grid, ModalOrder<3>::NT, ModalOrder<3>::bytes, s>>>(a); break;
    default: stage_modal_kernel<4><<<grid, ModalOrder<4>::NT, ModalOrder<4>::bytes, s>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace dgk
