// Learned boundary closure: a 12 -> 64 -> 64 -> 5 tanh network that maps
// what leaves the domain at an outer-face node to the acoustic wave that
// enters it (a learned impedance). All float32.
//
// Features of a face node with interior perturbation trace q'-, outward
// normal n, position x (R = radius used to scale positions) and memory psi
// of past outgoing waves (d psi/dt = -(c0 / 2|x|)(psi + w_out), the exact
// incoming invariant of an outgoing spherical wave), built from the parts of
// the trace the interior determines -- the outgoing acoustic invariant
// w_out = p' + rho0 c0 u.n, the entropy mode and the tangential velocity --
// and not from the incoming invariant (which the condition sets):
//   s    = (|w_out| + |psi|) / (rho0 c0^2) + 1e-12            (amplitude)
//   feat = (w_out / (rho0 c0^2 s),  (rho' - p'/c0^2) / (rho0 s),
//           u_t / (c0 s) (3),  n (3),  x / R (3),  psi / (rho0 c0^2 s))  (12 values)
// Output 0 is the incoming invariant the condition sets, relative to the
// memory psi (the spherical-wave value), in units of rho0 c0^2 s; outputs
// 1..4 are unused. A zero output layer gives the spherical-wave condition.
// The normalised perturbation z = (rho'/rho0, m'/(rho0 c0), E'/(rho0 c0^2))
// is kept for the trace diagnostics.
// Parameter packing (row-major, input index first):
//   W1[12][64], b1[64], W2[64][64], b2[64], W3[64][5], b3[5]   (5317 floats)
#pragma once
#include <cmath>
#include <cstdint>

namespace dgk {
namespace mlp {

constexpr int kIn = 12, kH = 64, kOut = 5;
constexpr int oW1 = 0;
constexpr int oB1 = oW1 + kIn * kH;
constexpr int oW2 = oB1 + kH;
constexpr int oB2 = oW2 + kH * kH;
constexpr int oW3 = oB2 + kH;
constexpr int oB3 = oW3 + kH * kOut;
constexpr int kParams = oB3 + kOut;   // 5317
// forward_smem reads every block of four with one 16-byte load
static_assert(oB1 % 4 == 0 && oW2 % 4 == 0 && oB2 % 4 == 0 && oW3 % 4 == 0 && kH % 4 == 0,
              "parameter blocks must start on 16-byte boundaries");

struct Scales {
  float rho0, c0, p0, gm1, inv_R;
  float r_floor;              // distance floor of the memory rate (1e-3 R)
};

// z of a perturbation state
__host__ __device__ inline void normalise(const float q[5], const Scales& S, float z[5]) {
  const float mref = S.rho0 * S.c0, eref = S.rho0 * S.c0 * S.c0;
  z[0] = q[0] / S.rho0;
  z[1] = q[1] / mref;
  z[2] = q[2] / mref;
  z[3] = q[3] / mref;
  z[4] = q[4] / eref;
}

__host__ __device__ inline void denormalise(const float z[5], const Scales& S, float q[5]) {
  const float mref = S.rho0 * S.c0, eref = S.rho0 * S.c0 * S.c0;
  q[0] = z[0] * S.rho0;
  q[1] = z[1] * mref;
  q[2] = z[2] * mref;
  q[3] = z[3] * mref;
  q[4] = z[4] * eref;
}

// features of a face node with memory psi; returns the amplitude s
__host__ __device__ inline float features(const float qm[5], const float n[3], const float x[3],
                                          float psi, const Scales& S, float feat[kIn]) {
  const float rinv = 1.0f / (S.rho0 + qm[0]);
  const float pp = S.gm1 * (qm[4] - 0.5f * (qm[1] * qm[1] + qm[2] * qm[2] + qm[3] * qm[3]) * rinv);
  const float u[3] = {qm[1] * rinv, qm[2] * rinv, qm[3] * rinv};
  const float un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  const float pref = S.rho0 * S.c0 * S.c0;
  const float wout = pp + S.rho0 * S.c0 * un;
  const float s = (fabsf(wout) + fabsf(psi)) / pref + 1e-12f;
  feat[0] = wout / (pref * s);
  feat[1] = (qm[0] - pp / (S.c0 * S.c0)) / (S.rho0 * s);
  for (int d = 0; d < 3; ++d) feat[2 + d] = (u[d] - un * n[d]) / (S.c0 * s);
  for (int d = 0; d < 3; ++d) feat[5 + d] = n[d];
  for (int d = 0; d < 3; ++d) feat[8 + d] = x[d] * S.inv_R;
  feat[11] = psi / (pref * s);
  return s;
}

// d psi / dt of the memory at distance r from the origin
__host__ __device__ inline float memory_rate(float psi, float wout, float r, const Scales& S) {
  return -(S.c0 / (2.0f * r)) * (psi + wout);
}

// tanh from the identity tanh(x) = 1 - 2 / (1 + e^{2x}), with e^{2x} =
// 2^{2x log2 e} from the hardware exp2 and the 2-ulp reciprocal: absolute
// error ~1e-7 (what matters for a hidden unit, which enters the next layer
// through a weighted sum); saturates to +-1 for large |x| (e^{2x} -> inf or 0).
__device__ __forceinline__ float tanh_fast(float x) {
  const float e = exp2f(x * 2.8853900817779268f);        // 2 log2(e)
  return 1.0f - __fdividef(2.0f, 1.0f + e);
}

// acc += a * b on two packed float32 lanes (one instruction for two FMAs)
__device__ __forceinline__ void fma2(uint64_t& acc, uint64_t a, uint64_t b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ uint64_t dup2(float x) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lo2(uint64_t v) { return __uint_as_float(uint32_t(v)); }
__device__ __forceinline__ float hi2(uint64_t v) { return __uint_as_float(uint32_t(v >> 32)); }

// y = W3^T tanh(W2^T tanh(W1^T x + b1) + b2) + b3 with the parameters in
// shared memory (16-byte aligned, mlp packing): every thread of a block
// reads the same words. Hidden units go in groups of eight, two per packed
// float32x2 FMA; outputs [0, NOUT) are formed (NOUT = 1: the closure's only
// output).
template <int NOUT>
__device__ inline void forward_smem(const float* __restrict__ sw, const float x[kIn],
                                    float y[NOUT]) {
  uint64_t xx[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) xx[i] = dup2(x[i]);
  float h1[kH];
#pragma unroll
  for (int j = 0; j < kH; j += 8) {
    const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(sw + oB1 + j);
    const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(sw + oB1 + j + 4);
    uint64_t a[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
      const ulonglong2 w0 = *reinterpret_cast<const ulonglong2*>(sw + oW1 + i * kH + j);
      const ulonglong2 w1 = *reinterpret_cast<const ulonglong2*>(sw + oW1 + i * kH + j + 4);
      fma2(a[0], w0.x, xx[i]);
      fma2(a[1], w0.y, xx[i]);
      fma2(a[2], w1.x, xx[i]);
      fma2(a[3], w1.y, xx[i]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h1[j + 2 * k] = tanh_fast(lo2(a[k]));
      h1[j + 2 * k + 1] = tanh_fast(hi2(a[k]));
    }
  }
  float out[NOUT];
#pragma unroll
  for (int o = 0; o < NOUT; ++o) out[o] = sw[oB3 + o];
#pragma unroll 1
  for (int j = 0; j < kH; j += 8) {
    const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(sw + oB2 + j);
    const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(sw + oB2 + j + 4);
    uint64_t a[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
    for (int i = 0; i < kH; ++i) {
      const uint64_t hh = dup2(h1[i]);
      const ulonglong2 w0 = *reinterpret_cast<const ulonglong2*>(sw + oW2 + i * kH + j);
      const ulonglong2 w1 = *reinterpret_cast<const ulonglong2*>(sw + oW2 + i * kH + j + 4);
      fma2(a[0], w0.x, hh);
      fma2(a[1], w0.y, hh);
      fma2(a[2], w1.x, hh);
      fma2(a[3], w1.y, hh);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float h2a = tanh_fast(lo2(a[k])), h2b = tanh_fast(hi2(a[k]));
#pragma unroll
      for (int o = 0; o < NOUT; ++o) {
        out[o] += h2a * sw[oW3 + (j + 2 * k) * kOut + o];
        out[o] += h2b * sw[oW3 + (j + 2 * k + 1) * kOut + o];
      }
    }
  }
#pragma unroll
  for (int o = 0; o < NOUT; ++o) y[o] = out[o];
}

}  // namespace mlp
}  // namespace dgk
