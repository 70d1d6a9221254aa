// Learned boundary closure on the tensor cores: the network 12 -> 64 -> 64
// (tanh) of every outer-face node of the learned boundary, per stage, as two
// batched GEMMs per tile of 128 nodes:
//
//   H1 = tanh(X W1 + b1)      X [128 x 12 (padded to 16)], W1 [12 x 64]
//   H2 = tanh(H1 W2 + b2)     H1 [128 x 64],                W2 [64 x 64]
//   y0 = H2 W3[:, 0] + b3[0]  (64 FMAs per node in the epilogue)
//
// Both GEMMs run on tcgen05 (kind::tf32, float32 accumulators in tensor
// memory) in three products of tf32 heads and tails (x = hi + lo;
// A_hi B_hi + A_hi B_lo + A_lo B_hi), which keeps float32-level accuracy.
//
// Two threads per node row: thread (row r, half h) reads accumulator columns
// 32h .. 32h + 31 of lane r (warps w and w + 4 share lane quadrant w mod 4)
// and handles hidden units 32h .. 32h + 31. The first GEMM accumulates in
// tensor-memory columns 0..63, the second in 64..127; the second runs as two
// K-halves through one 32-column operand buffer (half 0's units, then half
// 1's, re-read from columns 0..63), which the first GEMM's operand overlays.
// So a CTA needs ~73 KB of shared memory, no thread holds a row of hidden
// units in registers, and three CTAs (24 warps) share an SM. The h = 0
// thread of a row forms the node's features, and at the end
// combines the two halves of y0 and applies the closure: the incoming
// invariant psi + rho0 c0^2 s y0, bounded, as the increment D over the
// characteristic ghost's, and the memory psi's Runge-Kutta update. The
// weights' operand images are built once per weight change and copied into
// each CTA's shared memory; CTAs loop over tiles.
#include <cmath>

#include "cp_async.cuh"
#include "dg_device.cuh"
#include "ghost_f32.cuh"
#include "tc_ptx.cuh"

namespace dgk {

namespace {

constexpr int kRows = 128;                                 // node rows of a tile
constexpr int kCT = 2 * kRows;                             // threads: two per row
constexpr int kK1 = 16;                                    // layer-1 K: 12 features, padded
constexpr int kH = mlp::kH;                                // 64 hidden units
constexpr int kHH = kH / 2;                                // units of one half
constexpr uint32_t kSBO1 = uint32_t(kK1 / 4) * 128u;       // operand row-group strides
constexpr uint32_t kSBOh = uint32_t(kHH / 4) * 128u;       // layer-2 A (one K-half)
constexpr uint32_t kSBO2 = uint32_t(kH / 4) * 128u;        // layer-2 B (whole K)
constexpr uint32_t kA1 = uint32_t(kRows / 8) * kSBO1;      // bytes of one head or tail image
constexpr uint32_t kA2 = uint32_t(kRows / 8) * kSBOh;
constexpr uint32_t kB1 = uint32_t(kH / 8) * kSBO1;
constexpr uint32_t kB2 = uint32_t(kH / 8) * kSBO2;
static_assert(kA1 <= kA2, "the layer-1 operand overlays the layer-2 operand");
constexpr uint32_t oA2 = 0;                                // hi, then lo
constexpr uint32_t oA1 = oA2;                              // dead once layer 1 completes
constexpr uint32_t oB1 = oA2 + 2 * kA2;
constexpr uint32_t oB2 = oB1 + 2 * kB1;
constexpr uint32_t oVec = oB2 + 2 * kB2;                   // b1[64], b2[64], w3[64], b3
// B1, B2 (head and tail) and the vectors form one contiguous image, built
// once per weight change (closure_image_kernel) and copied whole per CTA
constexpr uint32_t kImgBytes = (2 * kB1 + 2 * kB2 + (3 * kH + 1) * 4 + 15) / 16 * 16;
static_assert(oB2 == oB1 + 2 * kB1 && oVec == oB2 + 2 * kB2 && oB1 % 16 == 0, "one image");
constexpr uint32_t oPart = oB1 + kImgBytes;                // y0 of half 1 [128]
constexpr uint32_t oFm = oPart + kRows * 4;               // face-node map [4 Nfp], Nfp <= 15
constexpr uint32_t oBar = oFm + 64 * 4;
constexpr uint32_t kSmem = oBar + 16;                      // mbarrier, tensor-memory slot
static_assert(kSmem <= 75u * 1024u, "three CTAs per SM");
constexpr uint32_t kCols = 2 * kH;                         // tensor-memory columns: two accumulators
constexpr uint32_t kHintTries = 1u << 22;                  // bounded waits, 200 ns hint per try

// head and tail of four consecutive entries (row, 4c .. 4c + 3) of an operand
__device__ __forceinline__ void store4(unsigned char* base, uint32_t half, uint32_t off,
                                       const float x[4]) {
  float4 h, l;
  h.x = tc::to_tf32(x[0]);
  h.y = tc::to_tf32(x[1]);
  h.z = tc::to_tf32(x[2]);
  h.w = tc::to_tf32(x[3]);
  l.x = tc::to_tf32(x[0] - h.x);
  l.y = tc::to_tf32(x[1] - h.y);
  l.z = tc::to_tf32(x[2] - h.z);
  l.w = tc::to_tf32(x[3] - h.w);
  *reinterpret_cast<float4*>(base + off) = h;
  *reinterpret_cast<float4*>(base + half + off) = l;
}

// the three products of one GEMM (ksteps steps of K = 8), committed to the
// mbarrier; a_sbo / b_sbo: row-group strides of the two operands
__device__ __forceinline__ void gemm3(uint32_t tmem, uint32_t a, uint32_t a_half, uint32_t a_sbo,
                                      uint32_t b, uint32_t b_half, uint32_t b_sbo, int ksteps,
                                      uint32_t accumulate, uint32_t idesc, uint64_t* mbar) {
#pragma unroll 1
  for (int s = 0; s < ksteps; ++s) {
    const uint32_t off = 256u * s;
    const uint64_t ah = tc::smem_desc(a + off, 128u, a_sbo);
    const uint64_t al = tc::smem_desc(a + a_half + off, 128u, a_sbo);
    const uint64_t bh = tc::smem_desc(b + off, 128u, b_sbo);
    const uint64_t bl = tc::smem_desc(b + b_half + off, 128u, b_sbo);
    tc::mma_tf32(tmem, ah, bh, idesc, (s > 0 || accumulate) ? 1u : 0u);
    tc::mma_tf32(tmem, ah, bl, idesc, 1u);
    tc::mma_tf32(tmem, al, bh, idesc, 1u);
  }
  tc::mma_commit(mbar);
}

// every warp waits for the current phase: lane 0 polls, the warp follows
__device__ __forceinline__ bool warp_wait(uint64_t* mbar, uint32_t phase) {
  uint32_t ok = 0;
  if ((threadIdx.x & 31) == 0) ok = tc::mbar_wait_hint(mbar, phase, kHintTries, 200u) ? 1u : 0u;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// The weight image from the parameter vector w: B1[j][i] = W1[i][j] (i < 12,
// zero to 16) and B2[j][i] = W2[i][j] in the operand layout (the hidden unit
// is the operand row, the input the K index), each as tf32 head and tail,
// then b1, b2, w3[:, 0] (output 0 only) and b3. One thread per entry;
// consecutive threads read consecutive entries of a row of W.
__global__ void closure_image_kernel(const float* __restrict__ w, unsigned char* __restrict__ img) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int n1 = kH * kK1, n2 = kH * kH;
  float* vec = reinterpret_cast<float*>(img + 2 * kB1 + 2 * kB2);
  if (t < n1 + n2) {
    const bool first = t < n1;
    const int u = first ? t : t - n1;
    const int i = u / kH, j = u - (u / kH) * kH;
    const float x = first ? (i < mlp::kIn ? w[mlp::oW1 + i * kH + j] : 0.0f) : w[mlp::oW2 + i * kH + j];
    const float h = tc::to_tf32(x);
    const uint32_t off = first ? tc::kmajor_offset(j, i, kSBO1) : 2 * kB1 + tc::kmajor_offset(j, i, kSBO2);
    const uint32_t half = first ? kB1 : kB2;
    *reinterpret_cast<float*>(img + off) = h;
    *reinterpret_cast<float*>(img + off + half) = tc::to_tf32(x - h);
  } else if (t < n1 + n2 + kH) {
    const int j = t - n1 - n2;
    vec[j] = w[mlp::oB1 + j];
    vec[kH + j] = w[mlp::oB2 + j];
    vec[2 * kH + j] = w[mlp::oW3 + j * mlp::kOut];
  } else if (t == n1 + n2 + kH) {
    vec[3 * kH] = w[mlp::oB3];
  }
}

// tanh(accumulator + bias) of 16 consecutive columns of this thread's lane
__device__ __forceinline__ void tanh16(uint32_t taddr, const float* bias, float (&h)[16]) {
  float d[16];
  tc::tmem_ld_32x32b_x16(taddr, d);
#pragma unroll
  for (int j = 0; j < 16; ++j) h[j] = mlp::tanh_fast(d[j] + bias[j]);
}

__global__ void __launch_bounds__(kCT, 3) closure_tc_kernel(ClosureArgs A, BaseGhost bg) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* vec = reinterpret_cast<float*>(smem + oVec);
  float* part = reinterpret_cast<float*>(smem + oPart);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + oBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + oBar + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kRows - 1), half = tid >> 7;      // warp w: lane quadrant w mod 4
  const bool net = A.w != nullptr;
  const int64_t total = A.nb * A.Nfp;
  const int ntiles = int((total + kRows - 1) / kRows);
  // the stage kernel launched after this one may take SMs as CTAs of this
  // grid finish and run its prologue; it waits for the whole grid before
  // its first tile
  griddep_launch_dependents();

  for (int j = tid; j < 4 * A.Nfp; j += kCT) reinterpret_cast<int32_t*>(smem + oFm)[j] = A.fmask[j];
  if (net) {
    // the weight image (B1, B2 head and tail, b1, b2, w3[:, 0], b3): 16-byte
    // copies, all in flight at once
    const uint4* src = reinterpret_cast<const uint4*>(A.wimg);
    for (int t = tid; t < int(kImgBytes / 16); t += kCT) cp_async16(smem + oB1 + 16 * t, src + t);
    cp_async_commit();
    if (tid == 0) {
      tc::mbar_init(mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      tc::tmem_alloc(tslot, kCols);
      tc::tmem_relinquish();
    }
    cp_async_wait_all();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = net ? *tslot : 0u;
  const uint32_t tq = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(kHH * half);
  const uint32_t sa = tc::smem_addr(smem);
  constexpr uint32_t idesc = tc::idesc_tf32(kRows, kH);
  const float pref = bg.rho0 * bg.c0 * bg.c0;
  uint32_t phase = 0;
  bool gave_up = false;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = int64_t(tile) * kRows + row;
    bool active = false;
    float qm[5] = {0, 0, 0, 0, 0}, nv[3] = {0, 0, 1}, xv[3] = {0, 0, 0}, psi = 0.0f;
    if (half == 0 && i < total) {
      // one dependent global load (the face slot) before the rest: the
      // trace, normal and connection all go out together; the mode test
      // only decides what is written back
      const int64_t slot = i / A.Nfp;
      const int m = int(i - slot * A.Nfp);
      xv[0] = A.bxyz[i * 3];
      xv[1] = A.bxyz[i * 3 + 1];
      xv[2] = A.bxyz[i * 3 + 2];
      psi = A.psi[i];
      const int32_t ef = A.bface[slot];
      const int64_t e = ef >> 2;
      const int f = ef & 3;
      const int nm = reinterpret_cast<const int32_t*>(smem + oFm)[f * A.Nfp + m];
      if (DG_IN(e >= 0 && e < A.K_all && nm >= 0 && nm < A.Np, A.status)) {
        const int32_t c = A.conn[e * 4 + f];
#pragma unroll
        for (int v = 0; v < 5; ++v) qm[v] = A.q[(e * 5 + v) * A.Np + nm];
        const float* g = A.geo + e * kGeoStride + kGeoNrm + 3 * f;
        nv[0] = g[0];
        nv[1] = g[1];
        nv[2] = g[2];
        active = c < 0 && A.bc_mode[(-1 - c) & 7] == 3;
      }
    }
    float wo_m = 0.0f, y0 = 0.0f, s = 0.0f, wi_c = 0.0f;
    if (half == 0) {
      float wi_m;
      acoustic_invariants(qm, nv, bg, wo_m, wi_m);
    }
    if (net) {
      if (half == 0) {
        float qc[5], wo_c;
        ghost_state_f(1, qm, nv, bg, qc);
        acoustic_invariants(qc, nv, bg, wo_c, wi_c);
        float feat[kK1];
        s = mlp::features(qm, nv, xv, psi, A.S, feat);
        for (int k = 0; k < kK1; ++k)
          if (k >= mlp::kIn || !active) feat[k] = 0.0f;
#pragma unroll
        for (int cq = 0; cq < kK1 / 4; ++cq)
          store4(smem + oA1, kA1, tc::kmajor_offset(row, 4 * cq, kSBO1), feat + 4 * cq);
      }
      // ---- layer 1: X W1 -> tensor memory columns 0..63
      tc::fence_smem_to_async();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        gemm3(tmem, sa + oA1, kA1, kSBO1, sa + oB1, kB1, kSBO1, kK1 / 8, 0u, idesc, mbar);
      }
      bool ok = warp_wait(mbar, phase);
      phase ^= 1u;
      tc::fence_after_sync();
      // ---- layer 2 in two K-halves through one operand buffer: the units
      // of half 0, then of half 1, each read from columns 0..63 (which the
      // second GEMM, accumulating in 64..127, leaves alone) when its turn comes
#pragma unroll 1
      for (int kh = 0; kh < 2; ++kh) {
        if (ok && half == kh) {
#pragma unroll
          for (int c16 = 0; c16 < kHH / 16; ++c16) {
            float h[16];
            tanh16(tq + uint32_t(16 * c16), vec + kHH * half + 16 * c16, h);
#pragma unroll
            for (int cq = 0; cq < 4; ++cq)
              store4(smem + oA2, kA2, tc::kmajor_offset(row, 16 * c16 + 4 * cq, kSBOh), h + 4 * cq);
          }
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        if (tid == 0) {
          tc::fence_after_sync();
          gemm3(tmem + uint32_t(kH), sa + oA2, kA2, kSBOh, sa + oB2 + 1024u * kh, kB2, kSBO2,
                kHH / 8, uint32_t(kh), idesc, mbar);
        }
        ok = warp_wait(mbar, phase);
        phase ^= 1u;
        tc::fence_after_sync();
      }
      float ypart = 0.0f;
      if (ok) {
#pragma unroll
        for (int c16 = 0; c16 < kHH / 16; ++c16) {
          float h[16];
          tanh16(tq + uint32_t(kH + 16 * c16), vec + kH + kHH * half + 16 * c16, h);
#pragma unroll
          for (int j = 0; j < 16; ++j) ypart += vec[2 * kH + kHH * half + 16 * c16 + j] * h[j];
        }
      }
      if (half == 1) part[row] = ypart;
      if (__syncthreads_or(!ok)) {
        // a completion wait gave up: report it, keep the characteristic
        // ghost (D = 0) on this tile and stop
        if (tid == 0) atomicOr(A.status, kStatusTimeout);
        gave_up = true;
      }
      y0 = vec[3 * kH] + ypart + (half == 0 ? part[row] : 0.0f);
    }
    if (half == 0 && active) {
      float D = 0.0f;
      if (net && !gave_up) {
        // the spherical-wave value psi plus the network's correction,
        // bounded by the characteristic ghost's own |w_in| or
        // |w_out| + |psi| (= rho0 c0^2 s), which holds psi
        const float lim = fmaxf(fabsf(wi_c), pref * s);
        D = fminf(fmaxf(psi + pref * s * y0, -lim), lim) - wi_c;
      }
      A.D[i] = D;
      if (A.advance) {
        const float r = fmaxf(sqrtf(xv[0] * xv[0] + xv[1] * xv[1] + xv[2] * xv[2]), A.S.r_floor);
        const float res = A.a * A.psi_res[i] + A.dt * mlp::memory_rate(psi, wo_m, r, A.S);
        A.psi_res[i] = res;
        A.psi[i] = psi + A.b * res;
      }
    }
    if (net) {
      tc::fence_before_sync();
      __syncthreads();                 // operands, partial sums and tensor memory free again
      if (gave_up) break;
    }
  }
  if (net) {
    // MMAs of a wait that gave up may still be in flight: a bounded chance to
    // finish (on the parity of that wait, phase ^ 1) before tensor memory is freed
    if (gave_up && tid == 0) tc::mbar_wait_hint(mbar, phase ^ 1u, kHintTries, 200u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
      tc::fence_after_sync();
      tc::tmem_dealloc(tmem, kCols);
    }
  }
}

}  // namespace

size_t closure_image_bytes() { return kImgBytes; }

cudaError_t launch_closure_image(const float* w, unsigned char* img, cudaStream_t s) {
  constexpr int n = kH * kK1 + kH * kH + kH + 1;
  closure_image_kernel<<<(n + 255) / 256, 256, 0, s>>>(w, img);
  return cudaGetLastError();
}

cudaError_t closure_prepare() {
  // the attributes belong to the current device: set by every context on it
  cudaError_t e = cudaFuncSetAttribute(closure_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(closure_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                              int(cudaSharedmemCarveoutMaxShared));
}

cudaError_t launch_closure(const ClosureArgs& A, const BaseGhost& bg, cudaStream_t s) {
  const int64_t total = A.nb * A.Nfp;
  if (total == 0) return cudaSuccess;
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (total + kRows - 1) / kRows;
  const int64_t want = 3 * int64_t(sms);                  // three CTAs per SM
  const int grid = int(ntiles < want ? ntiles : want);
  closure_tc_kernel<<<grid, kCT, kSmem, s>>>(A, bg);
  return cudaGetLastError();
}

}  // namespace dgk
