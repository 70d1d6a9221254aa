// Learned boundary closure: trace sampling, the per-stage closure and
// memory kernels, and the network's training kernels (forward, backward,
// Adam), all float32 on the device.
//
// Training data are traces the method records itself: at every node of a
// chosen set of interior faces (the truncation sphere inside a larger
// domain) the features of the inner trace and, as target, the part of the
// outer trace's incoming acoustic invariant that the spherical-wave memory
// psi misses (see mlp.cuh for the feature and target definitions).
//
// Loss: L = (1/N) sum_samples sum_outputs (y_pred - y)^2. Gradients come from
// hand-written backward passes over 64-sample chunks; every block owns a
// fixed set of chunks and every thread a fixed set of gradient entries, and
// the block partials are added in block order, so a gradient is the same on
// every run.
#include <cmath>

#include "dg_device.cuh"
#include "ghost_f32.cuh"

namespace dgk {

// ------------------------------------------------------------ trace sampling

__global__ void sample_traces_kernel(const float* __restrict__ q, int Np, int Nfp,
                                     const int32_t* __restrict__ tr_elem,
                                     const int8_t* __restrict__ tr_face,
                                     const int32_t* __restrict__ conn,
                                     const uint8_t* __restrict__ tbl,
                                     const int32_t* __restrict__ fmask,
                                     const float* __restrict__ geo, const float* __restrict__ txyz,
                                     const float* __restrict__ tr_psi, int64_t n, BaseGhost bg,
                                     mlp::Scales S, float* __restrict__ X, float* __restrict__ Y,
                                     float* __restrict__ amp, int* status) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n * Nfp) return;
  const int64_t t = i / Nfp;
  const int m = int(i - t * Nfp);
  const int64_t e = tr_elem[t];
  const int f = tr_face[t] & 3;
  const int32_t c = conn[e * 4 + f];
  if (c < 0) {                       // not an interior face: no outer trace to learn from
    atomicOr(status, kStatusBadState);
    return;
  }
  const int64_t e2 = c >> 5;
  const int f2 = (c >> 3) & 3, o = c & 7;
  const int nm = fmask[f * Nfp + m];
  const int np = tbl[((f * 4 + f2) * 6 + o) * Nfp + m];
  float qm[5], qo[5];
  for (int v = 0; v < 5; ++v) {
    qm[v] = q[(e * 5 + v) * Np + nm];
    qo[v] = q[(e2 * 5 + v) * Np + np];
  }
  const float* g = geo + e * kGeoStride + kGeoNrm + 3 * f;
  const float nv[3] = {g[0], g[1], g[2]};
  const float xv[3] = {txyz[i * 3], txyz[i * 3 + 1], txyz[i * 3 + 2]};
  float feat[mlp::kIn];
  const float s = mlp::features(qm, nv, xv, tr_psi[i], S, feat);
  float wo_o, wi_o;
  acoustic_invariants(qo, nv, bg, wo_o, wi_o);
  for (int k = 0; k < mlp::kIn; ++k) X[i * mlp::kIn + k] = feat[k];
  // target: what the outer trace's incoming invariant adds to the memory's
  // spherical-wave value psi, in units of rho0 c0^2 s; the other outputs are
  // not used by the closure and are trained towards zero
  Y[i * 5] = (wi_o - tr_psi[i]) / (bg.rho0 * bg.c0 * bg.c0 * s);
  for (int v = 1; v < 5; ++v) Y[i * 5 + v] = 0.0f;
  if (amp) amp[i] = bg.rho0 * bg.c0 * bg.c0 * s;
}

cudaError_t launch_sample_traces(const float* q, int Np, int Nfp, const int32_t* tr_elem,
                                 const int8_t* tr_face, const int32_t* conn, const uint8_t* tbl,
                                 const int32_t* fmask, const float* geo, const float* txyz,
                                 const float* tr_psi, int64_t n, const BaseGhost& bg,
                                 const mlp::Scales& S, float* X, float* Y, float* amp, int* status,
                                 cudaStream_t s) {
  const int64_t total = n * Nfp;
  if (total == 0) return cudaSuccess;
  sample_traces_kernel<<<unsigned((total + 127) / 128), 128, 0, s>>>(
      q, Np, Nfp, tr_elem, tr_face, conn, tbl, fmask, geo, txyz, tr_psi, n, bg, S, X, Y, amp,
      status);
  return cudaGetLastError();
}

// ------------------------------------------------------------ closure and memory
// (the closure itself runs on the tensor cores: closure_tc.cu)

__global__ void trace_memory_kernel(const float* __restrict__ q, int Np, int Nfp,
                                    const int32_t* __restrict__ tr_elem,
                                    const int8_t* __restrict__ tr_face,
                                    const int32_t* __restrict__ fmask,
                                    const float* __restrict__ geo, const float* __restrict__ txyz,
                                    int64_t n, BaseGhost bg, mlp::Scales S, float* __restrict__ psi,
                                    float* __restrict__ psi_res, float a, float b, float dt) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n * Nfp) return;
  const int64_t t = i / Nfp;
  const int m = int(i - t * Nfp);
  const int64_t e = tr_elem[t];
  const int f = tr_face[t] & 3;
  const int nm = fmask[f * Nfp + m];
  float qm[5];
  for (int v = 0; v < 5; ++v) qm[v] = q[(e * 5 + v) * Np + nm];
  const float* g = geo + e * kGeoStride + kGeoNrm + 3 * f;
  const float nv[3] = {g[0], g[1], g[2]};
  float wo, wi;
  acoustic_invariants(qm, nv, bg, wo, wi);
  const float x0 = txyz[i * 3], x1 = txyz[i * 3 + 1], x2 = txyz[i * 3 + 2];
  const float r = fmaxf(sqrtf(x0 * x0 + x1 * x1 + x2 * x2), S.r_floor);
  const float p = psi[i];
  const float res = a * psi_res[i] + dt * mlp::memory_rate(p, wo, r, S);
  psi_res[i] = res;
  psi[i] = p + b * res;
}

cudaError_t launch_trace_memory(const float* q, int Np, int Nfp, const int32_t* tr_elem,
                                const int8_t* tr_face, const int32_t* fmask, const float* geo,
                                const float* txyz, int64_t n, const BaseGhost& bg,
                                const mlp::Scales& S, float* psi, float* psi_res, float a,
                                float b, float dt, cudaStream_t s) {
  const int64_t total = n * Nfp;
  if (total == 0) return cudaSuccess;
  trace_memory_kernel<<<unsigned((total + 127) / 128), 128, 0, s>>>(
      q, Np, Nfp, tr_elem, tr_face, fmask, geo, txyz, n, bg, S, psi, psi_res, a, b, dt);
  return cudaGetLastError();
}

// ------------------------------------------------------------ network

namespace {
constexpr int kChunk = 64;          // samples per chunk
constexpr int kThreads = 256;
using namespace mlp;

// shared-memory layout of the gradient kernel (floats)
constexpr int sW_ = 0;
constexpr int sX_ = sW_ + kParams;
constexpr int sY_ = sX_ + kChunk * kIn;
constexpr int sH1_ = sY_ + kChunk * kOut;
constexpr int sH2_ = sH1_ + kChunk * kH;
constexpr int sD2_ = sH2_ + kChunk * kH;
constexpr int sD1_ = sD2_ + kChunk * kH;
constexpr int sDo_ = sD1_ + kChunk * kH;
constexpr int sAcc_ = sDo_ + kChunk * kOut;
constexpr int sLoss_ = sAcc_ + kParams;
constexpr int kGradSmemFloats = sLoss_ + kThreads;
}  // namespace

// Per block: loss and gradient summed over the block's chunks.
__global__ void __launch_bounds__(kThreads)
mlp_grad_kernel(const float* __restrict__ w, const float* __restrict__ X,
                const float* __restrict__ Y, int64_t N, float inv_n,
                float* __restrict__ part_grad, float* __restrict__ part_loss) {
  extern __shared__ float sm[];
  float* sW = sm + sW_;
  float* sX = sm + sX_;
  float* sY = sm + sY_;
  float* H1 = sm + sH1_;
  float* H2 = sm + sH2_;
  float* D2 = sm + sD2_;
  float* D1 = sm + sD1_;
  float* Do = sm + sDo_;
  float* acc = sm + sAcc_;
  float* sL = sm + sLoss_;
  const int tid = threadIdx.x;
  for (int i = tid; i < kParams; i += kThreads) {
    sW[i] = w[i];
    acc[i] = 0.0f;
  }
  float loss = 0.0f;
  const int64_t nchunks = (N + kChunk - 1) / kChunk;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t s0 = ch * kChunk;
    const int ns = int((N - s0) < kChunk ? (N - s0) : int64_t(kChunk));
    __syncthreads();
    for (int i = tid; i < kChunk * kIn; i += kThreads) sX[i] = (i / kIn < ns) ? X[s0 * kIn + i] : 0.0f;
    for (int i = tid; i < kChunk * kOut; i += kThreads) sY[i] = (i / kOut < ns) ? Y[s0 * kOut + i] : 0.0f;
    __syncthreads();
    // H1 = tanh(X W1 + b1)
    for (int i = tid; i < kChunk * kH; i += kThreads) {
      const int s = i / kH, j = i - (i / kH) * kH;
      float a = sW[oB1 + j];
      for (int k = 0; k < kIn; ++k) a += sX[s * kIn + k] * sW[oW1 + k * kH + j];
      H1[i] = tanh_fast(a);
    }
    __syncthreads();
    // H2 = tanh(H1 W2 + b2)
    for (int i = tid; i < kChunk * kH; i += kThreads) {
      const int s = i / kH, j = i - (i / kH) * kH;
      float a = sW[oB2 + j];
      for (int k = 0; k < kH; ++k) a += H1[s * kH + k] * sW[oW2 + k * kH + j];
      H2[i] = tanh_fast(a);
    }
    __syncthreads();
    // output, its error and the loss; dL/dout = 2 (out - y) / N
    for (int i = tid; i < kChunk * kOut; i += kThreads) {
      const int s = i / kOut, o = i - (i / kOut) * kOut;
      float a = sW[oB3 + o];
      for (int k = 0; k < kH; ++k) a += H2[s * kH + k] * sW[oW3 + k * kOut + o];
      const float d = (s < ns) ? a - sY[i] : 0.0f;
      loss += d * d;
      Do[i] = 2.0f * d * inv_n;
    }
    __syncthreads();
    // D2 = (Do W3^T) (1 - H2^2)
    for (int i = tid; i < kChunk * kH; i += kThreads) {
      const int s = i / kH, j = i - (i / kH) * kH;
      float a = 0.0f;
      for (int o = 0; o < kOut; ++o) a += Do[s * kOut + o] * sW[oW3 + j * kOut + o];
      D2[i] = a * (1.0f - H2[i] * H2[i]);
    }
    __syncthreads();
    // D1 = (D2 W2^T) (1 - H1^2)
    for (int i = tid; i < kChunk * kH; i += kThreads) {
      const int s = i / kH, j = i - (i / kH) * kH;
      float a = 0.0f;
      for (int k = 0; k < kH; ++k) a += D2[s * kH + k] * sW[oW2 + j * kH + k];
      D1[i] = a * (1.0f - H1[i] * H1[i]);
    }
    __syncthreads();
    // parameter gradients of this chunk; thread tid owns entries tid, tid + 256, ...
    for (int p = tid; p < kParams; p += kThreads) {
      float g = 0.0f;
      if (p < oB1) {                          // W1[k][j] += sum_s X[s][k] D1[s][j]
        const int k = p / kH, j = p - (p / kH) * kH;
        for (int s = 0; s < kChunk; ++s) g += sX[s * kIn + k] * D1[s * kH + j];
      } else if (p < oW2) {                   // b1[j]
        const int j = p - oB1;
        for (int s = 0; s < kChunk; ++s) g += D1[s * kH + j];
      } else if (p < oB2) {                   // W2[k][j] += sum_s H1[s][k] D2[s][j]
        const int q = p - oW2, k = q / kH, j = q - (q / kH) * kH;
        for (int s = 0; s < kChunk; ++s) g += H1[s * kH + k] * D2[s * kH + j];
      } else if (p < oW3) {                   // b2[j]
        const int j = p - oB2;
        for (int s = 0; s < kChunk; ++s) g += D2[s * kH + j];
      } else if (p < oB3) {                   // W3[k][o] += sum_s H2[s][k] Do[s][o]
        const int q = p - oW3, k = q / kOut, o = q - (q / kOut) * kOut;
        for (int s = 0; s < kChunk; ++s) g += H2[s * kH + k] * Do[s * kOut + o];
      } else {                                // b3[o]
        const int o = p - oB3;
        for (int s = 0; s < kChunk; ++s) g += Do[s * kOut + o];
      }
      acc[p] += g;
    }
  }
  __syncthreads();
  for (int p = tid; p < kParams; p += kThreads) part_grad[size_t(blockIdx.x) * kParams + p] = acc[p];
  sL[tid] = loss;
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f;
    for (int i = 0; i < kThreads; ++i) t += sL[i];
    part_loss[blockIdx.x] = t;
  }
}

// grad[p] = sum over blocks (in block order); loss likewise (times 1/N)
__global__ void mlp_reduce_kernel(const float* __restrict__ part_grad,
                                  const float* __restrict__ part_loss, int nblocks, float inv_n,
                                  float* __restrict__ grad, double* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kParams) {
    double g = 0.0;
    for (int b = 0; b < nblocks; ++b) g += double(part_grad[size_t(b) * kParams + p]);
    grad[p] = float(g);
  }
  if (p == 0) {
    double l = 0.0;
    for (int b = 0; b < nblocks; ++b) l += double(part_loss[b]);
    *loss = l * double(inv_n);
  }
}

// Adam step t (1-based) on every parameter
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, float lr, float beta1,
                            float beta2, float eps, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  const float g = grad[p];
  const float mm = beta1 * m[p] + (1.0f - beta1) * g;
  const float vv = beta2 * v[p] + (1.0f - beta2) * g * g;
  m[p] = mm;
  v[p] = vv;
  w[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
}

__global__ void __launch_bounds__(128)
mlp_forward_kernel(const float* __restrict__ w, const float* __restrict__ X, int64_t N,
                   float* __restrict__ out) {
  extern __shared__ __align__(16) float sw[];
  for (int k = threadIdx.x; k < kParams; k += blockDim.x) sw[k] = w[k];
  __syncthreads();
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float x[kIn], y[kOut];
  for (int k = 0; k < kIn; ++k) x[k] = X[i * kIn + k];
  mlp::forward_smem<kOut>(sw, x, y);
  for (int o = 0; o < kOut; ++o) out[i * kOut + o] = y[o];
}

int mlp_grad_blocks(int64_t N, int sms) {
  const int64_t chunks = (N + kChunk - 1) / kChunk;
  const int64_t b = chunks < int64_t(2 * sms) ? chunks : int64_t(2 * sms);
  return int(b < 1 ? 1 : b);
}

size_t mlp_grad_smem() { return size_t(kGradSmemFloats) * 4; }

cudaError_t mlp_prepare() {
  // the attribute belongs to the current device: set by every context on it
  return cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(mlp_grad_smem()));
}

cudaError_t launch_mlp_loss_grad(const float* w, const float* X, const float* Y, int64_t N,
                                 int nblocks, float* part_grad, float* part_loss, float* grad,
                                 double* loss, cudaStream_t s) {
  const float inv_n = 1.0f / float(N);
  mlp_grad_kernel<<<nblocks, kThreads, mlp_grad_smem(), s>>>(w, X, Y, N, inv_n, part_grad, part_loss);
  mlp_reduce_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(part_grad, part_loss, nblocks, inv_n, grad,
                                                          loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, const float* grad, float* m, float* v, float lr, int t,
                        cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.0f - std::pow(b1, float(t)), bc2 = 1.0f - std::pow(b2, float(t));
  adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(w, grad, m, v, lr, b1, b2, 1e-8f, bc1, bc2);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* w, const float* X, int64_t N, float* out,
                               cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  mlp_forward_kernel<<<unsigned((N + 127) / 128), 128, size_t(kParams) * 4, s>>>(w, X, N, out);
  return cudaGetLastError();
}

}  // namespace dgk
