// Pointwise Euler physics in float64 shared by the stage kernels: pressure
// and velocity from the conserved variables (Eq. 2), the normal Euler flux
// (Eq. 1) with the local wave speed, and the ghost states of outer faces
// (section 2.2 free stream, characteristic far field, section 2.3 wall).
#pragma once
#include <cmath>

#include "dg_device.cuh"

namespace dgk {

// 1/x by Newton-Raphson on f(y) = 1/y - x (y <- y + y (1 - x y)) from the
// hardware's approximate reciprocal: each step squares the relative error,
// so two steps take the estimate below double precision rounding (tested
// against the correctly rounded division to 2 ulp).
__device__ __forceinline__ double recip_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  y = fma(y, fma(-x, y, 1.0), y);
  y = fma(y, fma(-x, y, 1.0), y);
  return y;
}

// sqrt(x), x > 0: Newton-Raphson on 1/sqrt(x) (y <- y (3 - x y^2) / 2) from
// the hardware estimate, then s = x y and one Newton step on s
// (s <- s + (x - s^2) y / 2); 0 for x <= 0 (a non-physical state, which the
// kernels report separately). Tested against sqrt to 2 ulp.
__device__ __forceinline__ double sqrt_nr(double x) {
  if (!(x > 0.0)) return 0.0;
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  y = y * fma(-0.5 * x * y, y, 1.5);
  y = y * fma(-0.5 * x * y, y, 1.5);
  const double s = x * y;
  return fma(fma(-s, s, x), 0.5 * y, s);
}

__device__ __forceinline__ void pressure_and_velocity(const double q[5], double gm1, double& rinv,
                                                      double u[3], double& p) {
  rinv = recip_nr(q[0]);
  u[0] = q[1] * rinv;
  u[1] = q[2] * rinv;
  u[2] = q[3] * rinv;
  p = gm1 * (q[4] - 0.5 * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
}

// n.F(q) and |u.n| + c
__device__ __forceinline__ void normal_flux(const double q[5], const double n[3], const Gas& g,
                                            double fn[5], double& lam) {
  double rinv, u[3], p;
  pressure_and_velocity(q, g.gm1, rinv, u, p);
  const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  fn[0] = q[0] * un;
  fn[1] = q[1] * un + p * n[0];
  fn[2] = q[2] * un + p * n[1];
  fn[3] = q[3] * un + p * n[2];
  fn[4] = (q[4] + p) * un;
  lam = fabs(un) + sqrt_nr(g.gamma * p * rinv);
}

// Ghost state of an outer face node.
__device__ inline void ghost_state(int mode, const double qm[5], const double n[3], const Gas& g,
                            const double inflow[3], double qp[5]) {
  if (mode == 4) {  // inflow pulse (section 2.4, Eq. 7): rho, rho u_in along -n, E
    qp[0] = inflow[0];
    qp[1] = -inflow[1] * n[0];
    qp[2] = -inflow[1] * n[1];
    qp[3] = -inflow[1] * n[2];
    qp[4] = inflow[2];
    return;
  }
  if (mode == 0) {  // free stream (the paper's pass-through ghost)
    qp[0] = g.rho0;
    qp[1] = g.rho0 * g.u0[0];
    qp[2] = g.rho0 * g.u0[1];
    qp[3] = g.rho0 * g.u0[2];
    qp[4] = g.E0;
    return;
  }
  double rinv, u[3], p;
  pressure_and_velocity(qm, g.gm1, rinv, u, p);
  const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  if (mode == 2) {  // reflective wall: mirror the normal velocity
    const double mn = qm[1] * n[0] + qm[2] * n[1] + qm[3] * n[2];
    qp[0] = qm[0];
    qp[1] = qm[1] - 2.0 * mn * n[0];
    qp[2] = qm[2] - 2.0 * mn * n[1];
    qp[3] = qm[3] - 2.0 * mn * n[2];
    qp[4] = qm[4];
    return;
  }
  // characteristic far field: Riemann invariants along n
  const double gam = g.gamma;
  const double c = sqrt(gam * p * rinv);
  const double un_inf = g.u0[0] * n[0] + g.u0[1] * n[1] + g.u0[2] * n[2];
  const double Rp = un + 2.0 * c / g.gm1;
  const double Rm = un_inf - 2.0 * g.c0 / g.gm1;
  const double unb = 0.5 * (Rp + Rm);
  const double cb = 0.25 * g.gm1 * (Rp - Rm);
  double s, ut[3];
  if (unb >= 0.0) {  // outflow: entropy and tangential velocity from inside
    s = p / pow(qm[0], gam);
    for (int d = 0; d < 3; ++d) ut[d] = u[d] - un * n[d];
  } else {
    s = g.s_inf;
    for (int d = 0; d < 3; ++d) ut[d] = g.u0[d] - un_inf * n[d];
  }
  const double rhob = pow(cb * cb / (gam * s), 1.0 / g.gm1);
  const double pb = rhob * cb * cb / gam;
  double ub[3];
  for (int d = 0; d < 3; ++d) ub[d] = ut[d] + unb * n[d];
  qp[0] = rhob;
  qp[1] = rhob * ub[0];
  qp[2] = rhob * ub[1];
  qp[3] = rhob * ub[2];
  qp[4] = pb / g.gm1 + 0.5 * rhob * (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
}

}  // namespace dgk
