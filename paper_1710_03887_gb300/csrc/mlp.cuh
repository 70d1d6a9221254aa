// Learned boundary closure: a 12 -> 64 -> 64 -> 5 tanh network that maps
// what leaves the domain at an outer-face node to the acoustic wave that
// enters it (a learned impedance). All float32.
//
// Features of a face node with interior perturbation trace q'-, outward
// normal n and position x (R = radius used to scale positions), built from
// the parts of the trace the interior determines -- the outgoing acoustic
// invariant w_out = p' + rho0 c0 u.n, the entropy mode and the tangential
// velocity -- and not from the incoming invariant (which the condition sets):
//   s    = |w_out| / (rho0 c0^2) + 1e-12                 (outgoing amplitude)
//   feat = (w_out / (rho0 c0^2 s),  (rho' - p'/c0^2) / (rho0 s),
//           u_t / (c0 s) (3),  n (3),  x / R (3),  10 w_out / (2 p0))  (12 values)
// Output 0 is the incoming invariant the condition sets, relative to the
// characteristic ghost's, in units of rho0 c0^2 s; outputs 1..4 are unused.
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

struct Scales {
  float rho0, c0, p0, gm1, inv_R;
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

// features of a face node; returns the outgoing amplitude s
__host__ __device__ inline float features(const float qm[5], const float n[3], const float x[3],
                                          const Scales& S, float feat[kIn]) {
  const float rinv = 1.0f / (S.rho0 + qm[0]);
  const float pp = S.gm1 * (qm[4] - 0.5f * (qm[1] * qm[1] + qm[2] * qm[2] + qm[3] * qm[3]) * rinv);
  const float u[3] = {qm[1] * rinv, qm[2] * rinv, qm[3] * rinv};
  const float un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  const float pref = S.rho0 * S.c0 * S.c0;
  const float wout = pp + S.rho0 * S.c0 * un;
  const float s = fabsf(wout) / pref + 1e-12f;
  feat[0] = wout / (pref * s);
  feat[1] = (qm[0] - pp / (S.c0 * S.c0)) / (S.rho0 * s);
  for (int d = 0; d < 3; ++d) feat[2 + d] = (u[d] - un * n[d]) / (S.c0 * s);
  for (int d = 0; d < 3; ++d) feat[5 + d] = n[d];
  for (int d = 0; d < 3; ++d) feat[8 + d] = x[d] * S.inv_R;
  feat[11] = 10.0f * wout / (2.0f * pref / (S.gm1 + 1.0f));   // 10 w_out / (2 p0), p0 = rho0 c0^2 / gamma
  return s;
}

// y = W3^T tanh(W2^T tanh(W1^T x + b1) + b2) + b3, weights read through the
// read-only path (every thread of a tile reads the same parameters)
__device__ inline void forward(const float* __restrict__ w, const float x[kIn], float y[kOut]) {
  float h1[kH];
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float a = __ldg(w + oB1 + j);
#pragma unroll
    for (int i = 0; i < kIn; ++i) a += x[i] * __ldg(w + oW1 + i * kH + j);
    h1[j] = tanhf(a);
  }
  float out[kOut];
  for (int o = 0; o < kOut; ++o) out[o] = __ldg(w + oB3 + o);
#pragma unroll 2
  for (int j = 0; j < kH; ++j) {
    float a = __ldg(w + oB2 + j);
#pragma unroll 8
    for (int i = 0; i < kH; ++i) a += h1[i] * __ldg(w + oW2 + i * kH + j);
    const float h2 = tanhf(a);
#pragma unroll
    for (int o = 0; o < kOut; ++o) out[o] += h2 * __ldg(w + oW3 + j * kOut + o);
  }
  for (int o = 0; o < kOut; ++o) y[o] = out[o];
}

}  // namespace mlp
}  // namespace dgk
