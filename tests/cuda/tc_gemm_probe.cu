// Unit probe of the tensor-core building blocks in tc_ptx.cuh: one CTA
// computes D = A B^T (M = 128 rows, N columns, K a multiple of 8) with
// kind::tf32 MMAs from K-major shared-memory operands, accumulating in
// tensor memory, and writes D to global memory. Inputs are rounded to tf32
// on the device; status[0] is set when the MMA completion wait gives up.
#include <cstdint>

#include "../../paper_1710_03887_gb300/csrc/tc_ptx.cuh"

using namespace dgk;

__global__ void tc_gemm_probe_kernel(const float* A, const float* B, float* D, int N, int K,
                                     int* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int M = 128;
  const uint32_t sbo = uint32_t(K / 4) * 128u;
  float* As = reinterpret_cast<float*>(smem);
  float* Bs = reinterpret_cast<float*>(smem + size_t(M / 8) * sbo);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + size_t(M / 8 + N / 8) * sbo);
  uint32_t* slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < M * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    As[tc::kmajor_offset(r, k, sbo) / 4] = tc::to_tf32(A[i]);
  }
  for (int i = tid; i < N * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    Bs[tc::kmajor_offset(r, k, sbo) / 4] = tc::to_tf32(B[i]);
  }
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_smem_to_async();
  if (warp == 0) {
    tc::tmem_alloc(slot, 32);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *slot;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_tf32(M, N);
    const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs);
    for (int s = 0; s < K / 8; ++s) {
      const uint64_t ad = tc::smem_desc(a0 + 256u * s, 128u, sbo);
      const uint64_t bd = tc::smem_desc(b0 + 256u * s, 128u, sbo);
      tc::mma_tf32(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
    tc::mma_commit(mbar);
  }
  const bool ok = tc::mbar_wait(mbar, 0, 1u << 22);
  if (!ok && lane == 0) atomicOr(status, 1);
  tc::fence_after_sync();
  if (ok && warp < 4) {
    float v[32];
    tc::tmem_ld_32x32b_x32(taddr + (uint32_t(32 * warp) << 16), v);
    const int row = 32 * warp + lane;
    for (int j = 0; j < N; ++j) D[row * N + j] = v[j];
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 32);
  }
}

extern "C" int tc_gemm_probe(const float* A, const float* B, float* D, int N, int K, int* status) {
  if (N < 16 || N > 32 || N % 16 || K < 8 || K % 8 || K > 256) return -1;
  const size_t sbo = size_t(K / 4) * 128;
  const size_t bytes = size_t(128 / 8 + N / 8) * sbo + 16;
  if (cudaFuncSetAttribute(tc_gemm_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(bytes)) != cudaSuccess)
    return -2;
  tc_gemm_probe_kernel<<<1, 128, bytes>>>(A, B, D, N, K, status);
  if (cudaGetLastError() != cudaSuccess) return -3;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -4;
}

// The same product with M = 64 rows (instruction descriptor M field 64 >> 4):
// every lane of the 32-column allocation is read back into Dfull[128][32]
// (in bounds whatever the accumulator layout), so the host can locate the
// 64 result rows among the tensor-memory lanes.
__global__ void tc_gemm_probe_m64_kernel(const float* A, const float* B, float* Dfull, int N, int K,
                                         int* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int M = 64;
  const uint32_t sbo = uint32_t(K / 4) * 128u;
  float* As = reinterpret_cast<float*>(smem);
  float* Bs = reinterpret_cast<float*>(smem + size_t(M / 8) * sbo);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + size_t(M / 8 + (N + 7) / 8) * sbo);
  uint32_t* slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < M * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    As[tc::kmajor_offset(r, k, sbo) / 4] = tc::to_tf32(A[i]);
  }
  for (int i = tid; i < N * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    Bs[tc::kmajor_offset(r, k, sbo) / 4] = tc::to_tf32(B[i]);
  }
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_smem_to_async();
  if (warp == 0) {
    tc::tmem_alloc(slot, 32);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *slot;
  if (tid == 0) {
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) |
                           (uint32_t(M >> 4) << 24);
    const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs);
    for (int s = 0; s < K / 8; ++s) {
      const uint64_t ad = tc::smem_desc(a0 + 256u * s, 128u, sbo);
      const uint64_t bd = tc::smem_desc(b0 + 256u * s, 128u, sbo);
      tc::mma_tf32(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
    tc::mma_commit(mbar);
  }
  const bool ok = tc::mbar_wait(mbar, 0, 1u << 22);
  if (!ok && lane == 0) atomicOr(status, 1);
  tc::fence_after_sync();
  if (ok && warp < 4) {
    float v[32];
    tc::tmem_ld_32x32b_x32(taddr + (uint32_t(32 * warp) << 16), v);
    const int row = 32 * warp + lane;
    for (int j = 0; j < 32; ++j) Dfull[row * 32 + j] = v[j];
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 32);
  }
}

extern "C" int tc_gemm_probe_m64(const float* A, const float* B, float* Dfull, int N, int K,
                                 int* status) {
  if (N < 8 || N > 32 || N % 8 || K < 8 || K % 8 || K > 256) return -1;
  const size_t sbo = size_t(K / 4) * 128;
  const size_t bytes = size_t(64 / 8 + (N + 7) / 8) * sbo + 16;
  if (cudaFuncSetAttribute(tc_gemm_probe_m64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(bytes)) != cudaSuccess)
    return -2;
  tc_gemm_probe_m64_kernel<<<1, 128, bytes>>>(A, B, Dfull, N, K, status);
  if (cudaGetLastError() != cudaSuccess) return -3;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -4;
}

// ---- the network's tanh against CUDA's tanhf, elementwise
#include "../../paper_1710_03887_gb300/csrc/mlp.cuh"

__global__ void tanh_probe_kernel(const float* x, float* fast, float* ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  fast[i] = dgk::mlp::tanh_fast(x[i]);
  ref[i] = tanhf(x[i]);
}

extern "C" int tanh_probe(const float* x, float* fast, float* ref, int n) {
  if (n <= 0) return -1;
  tanh_probe_kernel<<<(n + 255) / 256, 256>>>(x, fast, ref, n);
  if (cudaGetLastError() != cudaSuccess) return -3;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -4;
}

// ---- bounded completion wait: an mbarrier nothing arrives at (no MMA is
// issued or committed) must give up after max_tries, report it in status,
// and still release its tensor memory
__global__ void tc_wait_timeout_kernel(uint32_t max_tries, int* status) {
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tc::tmem_alloc(&slot, 32);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = slot;
  uint32_t phase = 0;
  const bool ok = tc::mbar_wait(&mbar, phase, max_tries);
  if (!ok && tid == 0) atomicOr(status, 1);
  phase ^= 1u;                        // the stage kernel flips the parity after every wait
  if (tid == 0) {
    // the stage kernel's cleanup wait after a wait that gave up asks about
    // the parity that timed out (phase ^ 1): it must spin to its limit here,
    // since nothing ever completes that phase; the parity `phase` itself
    // names the phase before it, which counts as complete at once
    uint32_t used = 0;
    while (used < max_tries && !tc::mbar_try_wait(&mbar, phase ^ 1u)) ++used;
    status[1] = int(used);
    used = 0;
    while (used < max_tries && !tc::mbar_try_wait(&mbar, phase)) ++used;
    status[2] = int(used);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 32);
  }
}

extern "C" int tc_wait_timeout_probe(unsigned max_tries, int* status) {
  tc_wait_timeout_kernel<<<1, 128>>>(max_tries, status);
  if (cudaGetLastError() != cudaSuccess) return -3;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -4;
}

// ---- float64 reciprocal and square root of the float64 stage kernel
#include "../../paper_1710_03887_gb300/csrc/dg_physics.cuh"

__global__ void fp64_nr_probe_kernel(const double* x, double* rcp, double* rcp_ref, double* sq,
                                     double* sq_ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rcp[i] = dgk::recip_nr(x[i]);
  rcp_ref[i] = 1.0 / x[i];
  sq[i] = dgk::sqrt_nr(x[i]);
  sq_ref[i] = sqrt(x[i]);
}

extern "C" int fp64_nr_probe(const double* x, double* rcp, double* rcp_ref, double* sq,
                             double* sq_ref, int n) {
  if (n <= 0) return -1;
  fp64_nr_probe_kernel<<<(n + 255) / 256, 256>>>(x, rcp, rcp_ref, sq, sq_ref, n);
  if (cudaGetLastError() != cudaSuccess) return -3;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -4;
}
