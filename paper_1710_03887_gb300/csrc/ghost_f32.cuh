// Outer-face ghost states of the float32 perturbation form (resting free
// stream): the same rules as the float64 ghost_state (section 2.2 free
// stream, characteristic far field, section 2.3 wall), rewritten in
// quantities that stay small so nothing cancels against p0 or c0:
//   c - c0 = gamma (rho0 p' - p0 rho') / (rho rho0 (c + c0)),
//   u_n^b = u_n / 2 + (c - c0) / (gamma-1),  c_b - c0 = (gamma-1) u_n / 4 + (c - c0) / 2,
//   log(rho_b/rho0) = (2 log(c_b/c0) - log(s/s0)) / (gamma-1),
//   log(s/s0) = log(p/p0) - gamma log(rho/rho0)   (0 for inflow),
//   p_b - p0 = p0 expm1(log(rho_b/rho0) + 2 log(c_b/c0)).
// Mode 3 (learned) moves the characteristic ghost's incoming invariant by
// the closure kernel's increment and falls back to the characteristic ghost
// when the result is not finite or not physical.
#pragma once
#include <cmath>

#include "mlp.cuh"

namespace dgk {

struct BaseGhost {
  float rho0, p0, gamma, gm1, c0;
  // mode 4 (inflow pulse) at the stage time: rho - rho0, rho u_in (speed along
  // the inward normal), E - E0, formed on the host in float64
  float in_drho = 0.0f, in_m = 0.0f, in_dE = 0.0f;
};

__host__ __device__ inline void ghost_state_f(int mode, const float qm[5], const float n[3],
                                              const BaseGhost& g, float qp[5]) {
  if (mode == 0) {  // free stream: zero perturbation
    for (int v = 0; v < 5; ++v) qp[v] = 0.0f;
    return;
  }
  if (mode == 4) {  // inflow pulse (section 2.4, Eq. 7): the same state on every face
    qp[0] = g.in_drho;
    qp[1] = -g.in_m * n[0];
    qp[2] = -g.in_m * n[1];
    qp[3] = -g.in_m * n[2];
    qp[4] = g.in_dE;
    return;
  }
  if (mode == 2) {  // reflective wall
    const float mn = qm[1] * n[0] + qm[2] * n[1] + qm[3] * n[2];
    qp[0] = qm[0];
    qp[1] = qm[1] - 2.0f * mn * n[0];
    qp[2] = qm[2] - 2.0f * mn * n[1];
    qp[3] = qm[3] - 2.0f * mn * n[2];
    qp[4] = qm[4];
    return;
  }
  // characteristic far field (modes 1 and 3)
  const float rinv = 1.0f / (g.rho0 + qm[0]);
  const float u[3] = {qm[1] * rinv, qm[2] * rinv, qm[3] * rinv};
  const float pp = g.gm1 * (qm[4] - 0.5f * (qm[1] * u[0] + qm[2] * u[1] + qm[3] * u[2]));
  const float un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  const float c = sqrtf(g.gamma * (g.p0 + pp) * rinv);
  const float dc = g.gamma * (g.rho0 * pp - g.p0 * qm[0]) * rinv / (g.rho0 * (c + g.c0));
  const float unb = 0.5f * un + dc / g.gm1;
  const float dcb = 0.25f * g.gm1 * un + 0.5f * dc;
  const float lcb = log1pf(dcb / g.c0);                       // log(c_b / c0)
  float ls = 0.0f, ut[3] = {0.0f, 0.0f, 0.0f};
  if (unb >= 0.0f) {  // outflow: entropy and tangential velocity from inside
    ls = log1pf(pp / g.p0) - g.gamma * log1pf(qm[0] / g.rho0);
    for (int d = 0; d < 3; ++d) ut[d] = u[d] - un * n[d];
  }
  const float lrho = (2.0f * lcb - ls) / g.gm1;                // log(rho_b / rho0)
  const float drho = g.rho0 * expm1f(lrho);
  const float dp = g.p0 * expm1f(lrho + 2.0f * lcb);
  const float rhob = g.rho0 + drho;
  float ub[3];
  for (int d = 0; d < 3; ++d) ub[d] = ut[d] + unb * n[d];
  qp[0] = drho;
  qp[1] = rhob * ub[0];
  qp[2] = rhob * ub[1];
  qp[3] = rhob * ub[2];
  qp[4] = dp / g.gm1 + 0.5f * rhob * (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
}

// Acoustic invariants of a perturbation state along n (linearised about the
// resting free stream): w_out = p' + rho0 c0 u_n, w_in = p' - rho0 c0 u_n.
__host__ __device__ inline void acoustic_invariants(const float q[5], const float n[3],
                                                    const BaseGhost& g, float& w_out, float& w_in) {
  const float rinv = 1.0f / (g.rho0 + q[0]);
  const float pp = g.gm1 * (q[4] - 0.5f * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) * rinv);
  const float zun = g.rho0 * g.c0 * (q[1] * n[0] + q[2] * n[1] + q[3] * n[2]) * rinv;
  w_out = pp + zun;
  w_in = pp - zun;
}

// Learned closure at a face node. With a resting base state the local
// Lax-Friedrichs flux takes the outgoing acoustic invariant from inside and
// only the incoming one, g, from the ghost. The closure kernel (learned.cu)
// turns the network's output into the increment D = g - w_in(characteristic)
// of the incoming invariant, bounded by |g| <= max(|w_in(characteristic)|,
// |w_out| + |psi|); here the characteristic ghost is moved by D at fixed
// outgoing invariant (isentropic: d rho' = D / 2c0^2, d m' = -D n / 2c0,
// d E' = D / 2(gamma-1)). Non-finite or non-physical results fall back to
// the characteristic ghost.
__host__ __device__ inline void ghost_learned_f(const float qm[5], const float n[3],
                                                const BaseGhost& g, float D, float qp[5]) {
  ghost_state_f(1, qm, n, g, qp);
  if (D == 0.0f) return;
  float q[5];
  q[0] = qp[0] + D / (2.0f * g.c0 * g.c0);
  q[1] = qp[1] - D * n[0] / (2.0f * g.c0);
  q[2] = qp[2] - D * n[1] / (2.0f * g.c0);
  q[3] = qp[3] - D * n[2] / (2.0f * g.c0);
  q[4] = qp[4] + D / (2.0f * g.gm1);
  const float rho = g.rho0 + q[0];
  const float pp = g.gm1 * (q[4] - 0.5f * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / rho);
  bool ok = rho > 0.0f && g.p0 + pp > 0.0f;
  for (int v = 0; v < 5; ++v) ok = ok && isfinite(q[v]);
  if (ok)
    for (int v = 0; v < 5; ++v) qp[v] = q[v];
}

}  // namespace dgk
