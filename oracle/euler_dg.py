"""Nodal DG right-hand side and time step for 3D Euler (test infrastructure, float64).

What is computed, with the passage it follows:

* Conserved variables q = (rho, rho u, rho v, rho w, E) and the fluxes of the
  3D compressible Euler equations (section 2.1, Eq. 1), closed by the
  ideal-gas law E = p/(gamma-1) + rho |u|^2 / 2 (Eq. 2). Eq. 1 as printed has
  two typos (a "+p" in the z-momentum entry of the y-flux and in the
  y-momentum entry of the z-flux); the oracle uses the standard Euler fluxes,
  which is what Eq. 1 describes in words.
* Element-wise DG discretisation (Appendix A, Eqs. 8-12): for each element
      dq/dt = -(div F)_h + LIFT (Fscale * (n.F(q-) - F*)),
  i.e. the strong form of Eq. 10 obtained by integrating its volume term by
  parts back; on straight-sided elements with the nodal interpolant of the
  flux the two forms are the same discrete operator.
* Numerical flux on the shared face: local Lax-Friedrichs (section 1.1),
      F* = (n.F(q-) + n.F(q+))/2 - lambda (q+ - q-)/2,
      lambda = max(|u-.n| + c-, |u+.n| + c+) at each face node.
* Outer-boundary ghost states q+:
    FREESTREAM      the paper's pass-through condition: the ghost is the
                    initial (free-stream) state (section 2.2, Eq. 3);
    CHARACTERISTIC  Riemann-invariant far-field ghost (the characteristic
                    approach named in section 1 as the main far-field
                    technique): R+ = u.n + 2c/(g-1) from inside,
                    R- = u_inf.n - 2c_inf/(g-1) from the free stream; normal
                    velocity (R+ + R-)/2, sound speed (g-1)(R+ - R-)/4;
                    entropy p/rho^g and tangential velocity from inside when
                    that normal velocity is >= 0 (outflow), else from the
                    free stream;
    INFLOW_PULSE    the mouthpiece inflow of section 2.4 (Eqs. 5-7): a
                    time-dependent ghost (``ghost_inflow``);
    SLIP_WALL       reflective wall (section 2.3, Eq. 4): normal velocity
                    mirrored, rho and p unchanged. Eq. 4 as printed mixes
                    components (u - 2 u n_x, ...); the oracle mirrors the
                    normal component, u+ = u- - 2 (u-.n) n, which is what the
                    text around Eq. 4 states.
    LEARNED         not in the paper: the characteristic ghost with its
                    incoming acoustic invariant set to the spherical-wave
                    memory psi plus a network's correction, within a bound
                    (``ghost_learned``); the network is oracle/mlp.py.
* Time integration of the ODE system dc/dt = f(c) (Eq. 12) by the five-stage
  2N-storage fourth-order Runge-Kutta scheme of Carpenter and Kennedy (1994)
  instead of the paper's RK2 (section 1.1), stage by stage:
      res <- a_k res + dt f(q, t + c_k dt);  q <- q + b_k res.
* Sensors (section 3): point values of the five conserved variables through
  the element's interpolant.
* Boundary-flux ledger: the integral over outer faces of F*.n, integrated in
  time by the same stages, so that total(t) - total(0) + ledger(t) = 0.

Parity status: pinned (tests/test_oracle_euler.py: flux consistency and
antisymmetry, the LLF coefficient as the larger spectral radius of the two
flux Jacobians, free-stream preservation, discrete conservation, p+1
convergence against exact solutions, axis-permutation and inversion
symmetry, independence of the element vertex order, LSRK order conditions,
the characteristic ghost on 1D states and on an outgoing shear wave, a
plane simple wave leaving through it, the inflow ghost's free stream
outside its single pulse and its first-order plane-wave flux, the
contraction inputs recombining to the right-hand side, the probes' tie
rule; tests/test_oracle_mlp.py: the learned ghost's reduction to the
characteristic one and its bound, the memory against the closed form of an
outgoing spherical wave and its decay on the free stream). Planted mistakes
in every part of it make one of these fail
(tests/test_oracle_pins_catch_mistakes.py).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from .geometry import Geometry, inscribed_radius

FREESTREAM = 0
CHARACTERISTIC = 1
SLIP_WALL = 2
LEARNED = 3        # characteristic ghost + network correction (oracle/mlp.py)
INFLOW_PULSE = 4   # the mouthpiece pulse of section 2.4 (Eqs. 5-7)

# Carpenter & Kennedy (1994), NASA TM-109112, five-stage 2N-storage RK4
LSRK_A = [Fraction(0), Fraction(-567301805773, 1357537059087),
          Fraction(-2404267990393, 2016746695238),
          Fraction(-3550918686646, 2091501179385),
          Fraction(-1275806237668, 842570457699)]
LSRK_B = [Fraction(1432997174477, 9575080441755),
          Fraction(5161836677717, 13612068292357),
          Fraction(1720146321549, 2090206949498),
          Fraction(3134564353537, 4481467310338),
          Fraction(2277821191437, 14882151754819)]
LSRK_C = [Fraction(0), Fraction(1432997174477, 9575080441755),
          Fraction(2526269341429, 6820363962896),
          Fraction(2006345519317, 3224310063776),
          Fraction(2802321613138, 2924317926251)]


class Gas:
    """Ideal gas with a free stream (rho_inf, u_inf, p_inf)."""

    def __init__(self, gamma, rho0, p0, u0=(0.0, 0.0, 0.0)):
        self.gamma = float(gamma)
        self.rho0 = float(rho0)
        self.p0 = float(p0)
        self.u0 = np.asarray(u0, dtype=np.float64)
        self.c0 = np.sqrt(self.gamma * self.p0 / self.rho0)
        self.E0 = self.p0 / (self.gamma - 1.0) + 0.5 * self.rho0 * float(self.u0 @ self.u0)

    def freestream(self):
        return np.array([self.rho0, *(self.rho0 * self.u0), self.E0])


# ---------------------------------------------------------------- Eqs. 1-2

def pressure(q, gamma):
    """p from conserved variables (Eq. 2); q has the 5 variables on axis -1."""
    rho = q[..., 0]
    m = q[..., 1:4]
    return (gamma - 1.0) * (q[..., 4] - 0.5 * np.sum(m * m, axis=-1) / rho)


def euler_fluxes(q, gamma):
    """x, y, z fluxes of Eq. 1 (standard form); q[..., 5] -> three arrays [..., 5]."""
    rho = q[..., 0]
    u = q[..., 1:4] / rho[..., None]
    p = pressure(q, gamma)
    E = q[..., 4]
    out = []
    for d in range(3):
        f = np.empty_like(q)
        f[..., 0] = q[..., 1 + d]
        for e in range(3):
            f[..., 1 + e] = q[..., 1 + e] * u[..., d] + (p if d == e else 0.0)
        f[..., 4] = u[..., d] * (E + p)
        out.append(f)
    return out


def normal_flux(q, n, gamma):
    F, G, H = euler_fluxes(q, gamma)
    return n[..., 0:1] * F + n[..., 1:2] * G + n[..., 2:3] * H


def wave_speed(q, n, gamma):
    """|u.n| + c."""
    rho = q[..., 0]
    un = np.sum(q[..., 1:4] * n, axis=-1) / rho
    c = np.sqrt(gamma * pressure(q, gamma) / rho)
    return np.abs(un) + c


def llf_flux(qm, qp, n, gamma):
    """Local Lax-Friedrichs normal flux F*(q-, q+, n)."""
    lam = np.maximum(wave_speed(qm, n, gamma), wave_speed(qp, n, gamma))
    return 0.5 * (normal_flux(qm, n, gamma) + normal_flux(qp, n, gamma)) \
        - 0.5 * lam[..., None] * (qp - qm)


# ---------------------------------------------------------- ghost states

def ghost_freestream(qm, n, gas):
    return np.broadcast_to(gas.freestream(), qm.shape).copy()


def ghost_slip_wall(qm, n, gas):
    qp = qm.copy()
    mn = np.sum(qm[..., 1:4] * n, axis=-1)
    qp[..., 1:4] = qm[..., 1:4] - 2.0 * mn[..., None] * n
    return qp


def ghost_characteristic(qm, n, gas):
    g = gas.gamma
    rho = qm[..., 0]
    u = qm[..., 1:4] / rho[..., None]
    p = pressure(qm, g)
    c = np.sqrt(g * p / rho)
    un = np.sum(u * n, axis=-1)
    un_inf = np.sum(gas.u0 * n, axis=-1)
    Rp = un + 2.0 * c / (g - 1.0)
    Rm = un_inf - 2.0 * gas.c0 / (g - 1.0)
    unb = 0.5 * (Rp + Rm)
    cb = 0.25 * (g - 1.0) * (Rp - Rm)
    out = unb >= 0.0
    s_in = p / rho ** g
    s_inf = gas.p0 / gas.rho0 ** g
    s = np.where(out, s_in, s_inf)
    ut = np.where(out[..., None], u - un[..., None] * n,
                  gas.u0 - un_inf[..., None] * n)
    rhob = (cb * cb / (g * s)) ** (1.0 / (g - 1.0))
    pb = rhob * cb * cb / g
    ub = ut + unb[..., None] * n
    qp = np.empty_like(qm)
    qp[..., 0] = rhob
    qp[..., 1:4] = rhob[..., None] * ub
    qp[..., 4] = pb / (g - 1.0) + 0.5 * rhob * np.sum(ub * ub, axis=-1)
    return qp


def inflow_pressure(t, gas, amplitude, alpha):
    """Mouthpiece pressure of section 2.4: p0 (1 + A (1 - cos(alpha t))) while
    t < 2 pi / alpha (one unipolar pulse), p0 afterwards."""
    t = np.asarray(t, dtype=np.float64)
    on = (t >= 0.0) & (t < 2.0 * np.pi / alpha)
    return gas.p0 * (1.0 + np.where(on, amplitude * (1.0 - np.cos(alpha * t)), 0.0))


def ghost_inflow(qm, n, gas, t, amplitude, alpha):
    """Inflow ghost of section 2.4 (Eq. 7): the pulse pressure p(t), density
    from the adiabatic relation (Eq. 6) rho = rho0 (p/p0)^(1/gamma), and the
    velocity of a plane wave entering through the face (Eq. 5),
    (p - p0) / (rho0 c0) along the inward normal -n; E from Eq. 2. The paper
    states it for the bore's left end, where -n is +x."""
    p = inflow_pressure(t, gas, amplitude, alpha)
    rho = gas.rho0 * (p / gas.p0) ** (1.0 / gas.gamma)
    un = (p - gas.p0) / (gas.rho0 * gas.c0)
    q = np.zeros(qm.shape)
    q[..., 0] = rho
    q[..., 1:4] = -np.asarray(rho * un)[..., None] * n
    q[..., 4] = p / (gas.gamma - 1.0) + 0.5 * rho * un * un
    return q


GHOSTS = {FREESTREAM: ghost_freestream, CHARACTERISTIC: ghost_characteristic,
          SLIP_WALL: ghost_slip_wall}


def acoustic_invariants(qp, n, gas):
    """(w_out, w_in) = p' +- rho0 c0 u.n of perturbation states qp[..., 5]."""
    rho = gas.rho0 + qp[..., 0]
    pp = (gas.gamma - 1.0) * (qp[..., 4] - 0.5 * np.sum(qp[..., 1:4] ** 2, axis=-1) / rho)
    zun = gas.rho0 * gas.c0 * np.sum(qp[..., 1:4] * n, axis=-1) / rho
    return pp + zun, pp - zun


MEMORY_FLOOR = 1e-3      # r is floored at this fraction of the closure's scale R


def memory_rate(psi, wout, r, gas):
    """d psi / dt of the memory of an outer-face node at distance r from the
    origin: -(c0 / 2r) (psi + w_out).

    The asymptotic far-field route of section 1 (Bayliss and Turkel) in its
    lowest term: for an outgoing spherical wave of linear acoustics,
    p = f(t - r/c0) / r, the radial momentum equation integrates to
    rho0 c0 u_r = p + c0 F / r^2 with F the time integral of f, so at the node
    w_in = -c0 F / r^2 and w_out = 2 f / r + c0 F / r^2. Writing psi = -c0 F/r^2,
    dF/dt = f gives d psi/dt = -(c0/2r)(psi + w_out), and psi equals the
    incoming invariant of the exact solution exactly. The relation is a
    stable first-order filter of w_out (gain <= 1), so psi stays bounded."""
    return -(gas.c0 / (2.0 * r)) * (psi + wout)


def learned_target(qm, qo, n, psi, gas):
    """Training target of the closure at a face node with inner trace qm, outer
    trace qo (total states) and memory psi: what the outer trace's incoming
    acoustic invariant adds to the memory's spherical-wave value psi, in units
    of rho0 c0^2 s."""
    from . import mlp
    q0 = gas.freestream()
    _, s = mlp.features(qm - q0, n, np.zeros_like(n), psi, gas, 1.0)
    _, wi_o = acoustic_invariants(qo - q0, n, gas)
    y = np.zeros(qm.shape)
    y[..., 0] = (wi_o - psi) / (gas.rho0 * gas.c0 ** 2 * s)
    return y


def ghost_learned(qm, n, x, psi, gas, w, radius):
    """Learned closure. At rest the local Lax-Friedrichs flux takes the
    outgoing acoustic invariant w_out from inside and only the incoming one,
    g, from the ghost. The lowest-order far-field condition of section 1 for
    an outgoing spherical wave sets g to the node's memory psi
    (``memory_rate``); the network's output 0 corrects that value (in units of
    rho0 c0^2 s, s from the features with psi), so a network whose output
    layer is zero is the spherical-wave condition itself. The result is
    bounded by |g| <= L with L = max(|w_in(characteristic)|, |w_out(inside)| +
    |psi|), which holds psi; the characteristic ghost is moved to that
    invariant at fixed outgoing invariant (isentropic increments D/2c0^2,
    -D n/2c0, D/2(gamma-1), D = g - w_in(characteristic)). The
    characteristic ghost is kept where the result is not finite or has
    non-positive density or pressure."""
    from . import mlp
    q0 = gas.freestream()
    qc = ghost_characteristic(qm, n, gas)
    feats, s = mlp.features(qm - q0, n, x, psi, gas, radius)
    y, _ = mlp.forward(w, feats.reshape(-1, mlp.N_IN))
    y = y.reshape(qm.shape)
    _, wi_c = acoustic_invariants(qc - q0, n, gas)
    pref = gas.rho0 * gas.c0 ** 2
    lim = np.maximum(np.abs(wi_c), pref * s)
    D = np.clip(psi + pref * s * y[..., 0], -lim, lim) - wi_c
    c0 = gas.c0
    q = qc.copy()
    q[..., 0] += D / (2 * c0 * c0)
    q[..., 1:4] -= (D / (2 * c0))[..., None] * n
    q[..., 4] += D / (2 * (gas.gamma - 1.0))
    ok = np.all(np.isfinite(q), axis=-1) & (q[..., 0] > 0)
    ok &= pressure(np.where(ok[..., None], q, qc), gas.gamma) > 0
    return np.where(ok[..., None], q, qc)


# ----------------------------------------------------------------- solver

class Solver:
    """Semi-discrete DG operator plus time stepping on one mesh.

    ``bc_id[K, 4]`` gives a boundary id per face (ignored on interior faces;
    default 0 everywhere); ``bc_mode[id]`` the ghost rule of that id;
    ``mlp`` = (parameters, R) the network and position scale of the learned
    closure. Every node of a LEARNED face, and of the faces given to
    ``set_trace_faces``, carries a memory psi (``memory_rate``) integrated by
    the same Runge-Kutta stages as the state; ``step`` advances it in place
    and ``reset_memory`` (called by ``run``) zeroes it.
    """

    def __init__(self, geom: Geometry, gas: Gas, bc_id=None, bc_mode=None, mlp=None,
                 inflow=(0.05, 565.0)):
        self.g = geom
        self.inflow = inflow                # (amplitude A, rate alpha) of the mouthpiece pulse
        self.ref = geom.ref
        self.gas = gas
        self.mlp = mlp                      # (parameters, radius) of the learned closure
        self.radius = 1.0 if mlp is None else float(mlp[1])
        K = geom.K
        self.bc_id = np.zeros((K, 4), dtype=np.int64) if bc_id is None else np.asarray(bc_id)
        self.bc_mode = {0: CHARACTERISTIC} if bc_mode is None else dict(bc_mode)
        # physical face-integration weights of the face nodes: sJ * column sums of face mass
        self.face_w = np.stack([fm.sum(axis=0) for fm in self.ref.face_mass])  # [4, Nfp]
        # boundary faces grouped by id, in the order the right-hand side visits them
        self.groups = []
        mem_e, mem_f = [], []
        if np.any(geom.boundary):
            bidx = np.nonzero(geom.boundary)
            for ident in np.unique(self.bc_id[bidx]):
                sel = tuple(ix[self.bc_id[bidx] == ident] for ix in bidx)
                mode = self.bc_mode[int(ident)]
                row = None
                if mode == LEARNED:
                    if mlp is None:
                        raise ValueError("the learned closure needs mlp=(parameters, radius)")
                    row = sum(len(e) for e in mem_e)
                    mem_e.append(sel[0])
                    mem_f.append(sel[1])
                self.groups.append((mode, sel, row))
        self.n_learned = sum(len(e) for e in mem_e)
        self._set_memory_faces(mem_e, mem_f)

    def _set_memory_faces(self, mem_e, mem_f):
        g, ref = self.g, self.ref
        self.mem_elem = np.concatenate(mem_e).astype(np.int64) if mem_e else np.zeros(0, np.int64)
        self.mem_face = np.concatenate(mem_f).astype(np.int64) if mem_f else np.zeros(0, np.int64)
        x = g.x[self.mem_elem[:, None], ref.Fmask[self.mem_face]]          # [nmem, Nfp, 3]
        self.mem_x = x
        self.mem_r = np.maximum(np.linalg.norm(x, axis=-1), MEMORY_FLOOR * self.radius)
        self.reset_memory()

    def set_trace_faces(self, elem, face):
        """Interior faces (inner element, face) whose inner trace carries a memory
        too (the recording side of the learned closure); see ``trace_samples``."""
        le = [self.mem_elem[:self.n_learned], np.asarray(elem, dtype=np.int64)]
        lf = [self.mem_face[:self.n_learned], np.asarray(face, dtype=np.int64)]
        self._set_memory_faces(le, lf)

    def reset_memory(self):
        self.psi = np.zeros((len(self.mem_elem), self.ref.Nfp))
        self.psi_res = np.zeros_like(self.psi)

    # -- Eq. 10 / Eq. 12 right-hand side
    def rhs(self, q, t=0.0, want_ledger=False):
        out, ledger, _ = self.rhs_full(q, t, self.psi)
        return (out, ledger) if want_ledger else out

    def rhs_parts(self, q):
        """The inputs of the two contractions of Eq. 10 at state q: the
        metric-folded fluxes Ft [K, 3, 5, Np] (F~_r, F~_s, F~_t) and the face
        terms dF [K, 5, 4 Nfp], so that
        rhs = -(Dr Ft_r + Ds Ft_s + Dt Ft_t) + LIFT dF."""
        return self._rhs(q, self.psi, 0.0, parts=True)

    def rhs_full(self, q, t, psi):
        """(dq/dt, boundary flux integral, d psi/dt) at state q, time t, memory psi."""
        return self._rhs(q, psi, t)

    def _rhs(self, q, psi, t, parts=False):
        g, ref, gas = self.g, self.ref, self.gas
        gam = gas.gamma
        K, Np, Nfp = g.K, ref.Np, ref.Nfp
        qn = np.transpose(q, (0, 2, 1))                       # [K, Np, 5]
        F, G, H = euler_fluxes(qn, gam)
        flux = [np.transpose(f, (0, 2, 1)) for f in (F, G, H)]  # [K, 5, Np]
        D = [ref.Dr, ref.Ds, ref.Dt]
        div = np.zeros_like(q)
        for a in range(3):
            for b in range(3):
                dab = np.einsum("ij,kvj->kvi", D[a], flux[b])
                div += g.drdx[:, a, b][:, None, None] * dab
        if parts:
            Ft = np.stack([sum(g.drdx[:, a, b][:, None, None] * flux[b] for b in range(3))
                           for a in range(3)], axis=1)
        # face traces
        flat = qn.reshape(K * Np, 5)
        qm = flat[g.vmapM]                                    # [K, 4, Nfp, 5]
        qp = flat[g.vmapP].copy()
        n = np.broadcast_to(g.nrm[:, :, None, :], (K, 4, Nfp, 3))
        for mode, sel, row in self.groups:
            if mode == LEARNED:
                rows = slice(row, row + len(sel[0]))
                qp[sel] = ghost_learned(qm[sel], n[sel], self.mem_x[rows], psi[rows], gas,
                                        self.mlp[0], self.radius)
            elif mode == INFLOW_PULSE:
                qp[sel] = ghost_inflow(qm[sel], n[sel], gas, t, *self.inflow)
            else:
                qp[sel] = GHOSTS[mode](qm[sel], n[sel], gas)
        fstar = llf_flux(qm, qp, n, gam)
        dF = g.Fscale[:, :, None, None] * (normal_flux(qm, n, gam) - fstar)
        dF = np.transpose(dF, (0, 3, 1, 2)).reshape(K, 5, 4 * Nfp)
        if parts:
            return Ft, dF
        lift = np.einsum("ij,kvj->kvi", ref.LIFT, dF)
        out = -div + lift
        w = g.sJ[:, :, None] * self.face_w[None, :, :]        # [K, 4, Nfp]
        w = w * g.boundary[:, :, None]
        ledger = np.einsum("kfm,kfmv->v", w, fstar)
        # memory of the learned and trace faces, driven by the inner trace's w_out
        qmm = qm[self.mem_elem, self.mem_face] - gas.freestream()
        nm = np.broadcast_to(g.nrm[self.mem_elem, self.mem_face][:, None, :], qmm.shape[:2] + (3,))
        wout, _ = acoustic_invariants(qmm, nm, gas)
        dpsi = memory_rate(psi, wout, self.mem_r, gas)
        return out, ledger, dpsi

    # -- Eq. 12 integrated by the 2N-storage RK4
    def step(self, q, t, dt, res=None, ledger=None):
        """One full time step (the memory advances in place). Returns
        (q, t, res, (ledger, ledger_res))."""
        res = np.zeros_like(q) if res is None else res
        L = np.zeros(5) if ledger is None else ledger[0]
        Lres = np.zeros(5) if ledger is None else ledger[1]
        psi, pres = self.psi, self.psi_res
        for k in range(5):
            a, b, c = float(LSRK_A[k]), float(LSRK_B[k]), float(LSRK_C[k])
            rhs, lrhs, prhs = self.rhs_full(q, t + c * dt, psi)
            res = a * res + dt * rhs
            q = q + b * res
            Lres = a * Lres + dt * lrhs
            L = L + b * Lres
            pres = a * pres + dt * prhs
            psi = psi + b * pres
        self.psi, self.psi_res = psi, pres
        return q, t + dt, res, (L, Lres)

    def run(self, q, dt, nsteps, t=0.0, probes=None):
        """nsteps steps from q with zero memory; returns (q, t, ledger, probe
        samples [nsteps, n, 5])."""
        self.reset_memory()
        res = np.zeros_like(q)
        led = (np.zeros(5), np.zeros(5))
        samples = []
        for _ in range(nsteps):
            q, t, res, led = self.step(q, t, dt, res, led)
            if probes is not None:
                samples.append(probes.sample(q))
        return q, t, led[0], (np.array(samples) if probes is not None else None)

    def trace_samples(self, q):
        """Features [n, Nfp, 12], targets [n, Nfp, 5] and amplitudes s [n, Nfp]
        at the trace faces (the inner trace, its memory, and the outer trace
        as what the closure should have produced)."""
        from . import mlp
        g, ref, gas = self.g, self.ref, self.gas
        e, f = self.mem_elem[self.n_learned:], self.mem_face[self.n_learned:]
        psi = self.psi[self.n_learned:]
        flat = np.transpose(q, (0, 2, 1)).reshape(-1, 5)
        qm = flat[g.vmapM[e, f]]
        qo = flat[g.vmapP[e, f]]
        nv = np.broadcast_to(g.nrm[e, f][:, None, :], qm.shape[:2] + (3,))
        feats, s = mlp.features(qm - gas.freestream(), nv, self.mem_x[self.n_learned:], psi, gas,
                                self.radius)
        return feats, learned_target(qm, qo, nv, psi, gas), s

    # -- diagnostics
    def totals(self, q):
        """sum_e J_e 1^T M q_e for each conserved variable."""
        Mq = np.einsum("ij,kvj->kvi", self.ref.M, q)
        return np.einsum("k,kvi->v", self.g.J, Mq)

    def stable_dt(self, q, cfl=0.5):
        """CFL * min r_in / ((p+1)^2 * max(|u| + c)) at the given state."""
        qn = np.transpose(q, (0, 2, 1))
        rho = qn[..., 0]
        u = qn[..., 1:4] / rho[..., None]
        c = np.sqrt(self.gas.gamma * pressure(qn, self.gas.gamma) / rho)
        smax = np.max(np.linalg.norm(u, axis=-1) + c)
        p = self.ref.p
        return cfl * np.min(inscribed_radius(self.g)) / ((p + 1) ** 2 * smax)


class Probes:
    """Point sensors: element lookup and interpolation rows."""

    def __init__(self, geom: Geometry, pts, tol=1e-12):
        pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
        v = geom.verts
        self.elem = np.zeros(len(pts), dtype=np.int64)
        self.rows = np.zeros((len(pts), geom.ref.Np))
        for i, x in enumerate(pts):
            # barycentrics of x in every element: solve the affine map
            T = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
            lam = np.linalg.solve(T, (x - v[:, 0])[:, :, None])[:, :, 0]   # lam2..lam4
            lam1 = 1.0 - lam.sum(axis=1)
            inside = (lam.min(axis=1) >= -tol) & (lam1 >= -tol)
            hit = np.nonzero(inside)[0]
            if hit.size == 0:
                raise ValueError(f"probe {i} lies outside the mesh")
            e = hit[0]
            r, s, t = -1 + 2 * lam[e]
            self.elem[i] = e
            self.rows[i] = geom.ref.interp_row(r, s, t)[0]

    def sample(self, q):
        return np.einsum("pn,pvn->pv", self.rows, q[self.elem])
