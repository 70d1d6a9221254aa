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

// Device address of the scratch array, looked up once per device and
// context. The runtime gives host code only a stand-in for g_totals_scratch;
// the address comes from cudaGetSymbolAddress with the device current. A
// cudaDeviceReset destroys the primary context and the module with it, so the
// address is keyed on the context's process-unique id (cuCtxGetId, reached
// through the runtime's driver entry points) and looked up again when that id
// changes.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
  void* addr = nullptr;
  unsigned long long ctx_id = 0;
};
std::mutex g_mu;
ScratchSlot g_slot[kMaxDevices];

typedef int (*PfnCtxGetCurrent)(void** ctx);
typedef int (*PfnCtxGetId)(void* ctx, unsigned long long* id);
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
bool g_entry_points_tried = false;

// id of the current context, 0 when it cannot be told (no context yet, or a
// driver without the entry points)
unsigned long long current_ctx_id() {
  if (!g_entry_points_tried) {
    g_entry_points_tried = true;
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
      g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f2);
    }
  }
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
  if (g_ctx_get_id(ctx, &id) != 0) return 0;
  return id;
}

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
    ScratchSlot& slot = g_slot[dev];
    const unsigned long long id = slot.addr ? current_ctx_id() : 0;
    if (!slot.addr || id != slot.ctx_id) {
      // set-up for this device and context: the lookup also creates the
      // primary context if none is current yet
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_totals_scratch) != cudaSuccess || !addr) return DG_ERR_CUDA;
      slot.addr = addr;
      slot.ctx_id = current_ctx_id();
    }
    scratch = slot.addr;
  }
  const int nblocks = int((K + kElemsPerBlock - 1) / kElemsPerBlock);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* partial = static_cast<double*>(scratch);
  // cudaLaunchKernel returns the error of this launch itself, so an earlier
  // asynchronous error of the caller's is neither reported as ours nor
  // cleared from the thread's error state
  void* a1[] = {(void*)&q, (void*)&J, (void*)&w, (void*)&K, (void*)&Np, (void*)&partial};
  if (cudaLaunchKernel((const void*)static_totals_partial, dim3(nblocks), dim3(kThreads), a1, 0,
                       s) != cudaSuccess)
    return DG_ERR_CUDA;
  const double* cpartial = partial;
  void* a2[] = {(void*)&cpartial, (void*)&nblocks, (void*)&out};
  if (cudaLaunchKernel((const void*)static_totals_final, dim3(1), dim3(32), a2, 0, s) !=
      cudaSuccess)
    return DG_ERR_CUDA;
  return DG_OK;
}
