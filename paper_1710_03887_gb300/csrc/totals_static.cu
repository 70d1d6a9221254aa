// Conserved totals without any allocation: a variant of the library's
// two-pass totals reduction whose per-block partial sums live in a
// file-scope device array instead of a buffer the context allocates.
//
// For callers that cannot allocate device memory at the point where they
// need the totals: code whose device memory is entirely owned by another
// allocator (a framework's caching pool), and monitoring code inside a
// running time loop that must not call cudaMalloc/cudaFree, which can block
// or synchronise the device. Everything it touches is either passed in by
// the caller or the static array below.
#include <cstdint>
#include <mutex>

#include "../../include/dg_euler.h"

namespace {

constexpr int kBlocks = DG_STATIC_TOTALS_MAX_BLOCKS;          // partial sums
constexpr int64_t kElemsPerBlock = DG_STATIC_TOTALS_ELEMS_PER_BLOCK;
constexpr int kThreads = 256;

// Scratch shared by every call on a device: one 5-vector per block, each
// written by its block before the final pass reads it, so nothing needs to
// start at zero. 4096 x 5 doubles = 160 KiB per device that loads the library.
static __device__ __align__(256) double g_totals_scratch[kBlocks * 5];

__global__ void static_totals_partial(const double* __restrict__ q, const double* __restrict__ J,
                                      const double* __restrict__ w, int64_t K, int Np,
                                      double* __restrict__ partial) {
  __shared__ double red[kThreads * 5];
  const int tid = threadIdx.x;
  const int64_t lo = int64_t(blockIdx.x) * kElemsPerBlock;
  const int64_t hi = (lo + kElemsPerBlock < K) ? lo + kElemsPerBlock : K;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t e = lo + tid; e < hi; e += kThreads) {
    const double Je = J[e];
    for (int v = 0; v < 5; ++v) {
      const double* src = q + (e * 5 + v) * Np;
      double s = 0.0;
      for (int j = 0; j < Np; ++j) s += w[j] * src[j];
      acc[v] += Je * s;
    }
  }
  for (int v = 0; v < 5; ++v) red[tid * 5 + v] = acc[v];
  __syncthreads();
  for (int half = kThreads / 2; half > 0; half >>= 1) {
    if (tid < half)
      for (int v = 0; v < 5; ++v) red[tid * 5 + v] += red[(tid + half) * 5 + v];
    __syncthreads();
  }
  if (tid < 5) partial[blockIdx.x * 5 + tid] = red[tid];
}

__global__ void static_totals_final(const double* __restrict__ partial, int nblocks,
                                    double* __restrict__ out) {
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[b * 5 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" int dg_weighted_totals_static(const double* q, const double* J, const double* w,
                                         int64_t K, int Np, double* out, void* stream) {
  if (!q || !J || !w || !out) return DG_ERR_ARG;
  if (K <= 0 || K > DG_STATIC_TOTALS_MAX_ELEMENTS) return DG_ERR_ARG;
  if (Np < 1 || Np > DG_STATIC_TOTALS_MAX_NP) return DG_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return DG_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      // host code sees only a stand-in for g_totals_scratch; the device
      // address comes from the runtime, with this device current
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_totals_scratch) != cudaSuccess || !addr) return DG_ERR_CUDA;
      g_scratch_addr[dev] = addr;
    }
    scratch = g_scratch_addr[dev];
  }
  const int nblocks = int((K + kElemsPerBlock - 1) / kElemsPerBlock);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* partial = static_cast<double*>(scratch);
  static_totals_partial<<<nblocks, kThreads, 0, s>>>(q, J, w, K, Np, partial);
  static_totals_final<<<1, 32, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
