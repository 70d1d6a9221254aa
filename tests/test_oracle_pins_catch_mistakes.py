"""Strength of the oracle's pins: plausible mistakes are planted in the
oracle (on the CPU, through pytest's monkeypatch, undone after each case)
and each must make at least one of the named pins fail.

A pin that still passes with the mistake in place would not have caught it:
this is the evidence that the pins constrain every part of the oracle (a
dropped term, a wrong sign, index or factor, a transposed operand, a wrong
coefficient), not only its overall plausibility. Each case names the fast
pins that catch it; the slower pins (convergence rates, symmetry) catch
many of them as well.
"""
import functools
import sys

import numpy as np
import pytest

from oracle import euler_dg as ED
from oracle import geometry as GE
from oracle import mlp as ML
from oracle import modal_dg as MD
from oracle import reference_element as RE

from . import test_oracle_euler as E
from . import test_oracle_mlp as L
from . import test_oracle_modal as M
from . import test_oracle_reference as R


def _replace(mp, orig, new):
    """Replace a function everywhere the oracle and the pins hold a reference to it."""
    for name, mod in list(sys.modules.items()):
        if mod is None or not (name == "oracle" or name.startswith(("oracle.", "tests."))):
            continue
        for k, v in list(vars(mod).items()):
            if v is orig:
                mp.setattr(mod, k, new)
    for mode, fn in list(ED.GHOSTS.items()):
        if fn is orig:
            mp.setitem(ED.GHOSTS, mode, new)


def _after_init(mp, cls, post):
    orig = cls.__init__

    def init(self, *a, **kw):
        orig(self, *a, **kw)
        post(self)
    mp.setattr(cls, "__init__", init)


# ------------------------------------------------------------ the mistakes

def _flux_as_printed(mp):
    # Eq. 1 as printed: + p in the y-flux z-momentum and z-flux y-momentum rows
    orig = ED.euler_fluxes

    def bad(q, gamma):
        F, G, H = orig(q, gamma)
        p = ED.pressure(q, gamma)
        G, H = G.copy(), H.copy()
        G[..., 3] += p
        H[..., 2] += p
        return [F, G, H]
    _replace(mp, orig, bad)


def _pressure_factor(mp, which):
    orig = ED.pressure

    def bad(q, gamma):
        rho, m = q[..., 0], q[..., 1:4]
        if which == "gamma":
            return gamma * (q[..., 4] - 0.5 * np.sum(m * m, axis=-1) / rho)
        return (gamma - 1.0) * (q[..., 4] - np.sum(m * m, axis=-1) / rho)
    _replace(mp, orig, bad)


def _llf(mp, which):
    orig = ED.llf_flux

    def bad(qm, qp, n, gamma):
        a, b = ED.wave_speed(qm, n, gamma), ED.wave_speed(qp, n, gamma)
        lam = {"sign": -np.maximum(a, b), "min": np.minimum(a, b), "central": 0.0 * a}[which]
        return 0.5 * (ED.normal_flux(qm, n, gamma) + ED.normal_flux(qp, n, gamma)) \
            - 0.5 * lam[..., None] * (qp - qm)
    _replace(mp, orig, bad)


def _wave_speed_signed(mp):
    orig = ED.wave_speed

    def bad(q, n, gamma):
        un = np.sum(q[..., 1:4] * n, axis=-1) / q[..., 0]
        return un + np.sqrt(gamma * ED.pressure(q, gamma) / q[..., 0])
    _replace(mp, orig, bad)


def _slip_wall_half(mp):
    orig = ED.ghost_slip_wall

    def bad(qm, n, gas):
        qp = qm.copy()
        qp[..., 1:4] -= np.sum(qm[..., 1:4] * n, axis=-1)[..., None] * n
        return qp
    _replace(mp, orig, bad)


def _characteristic(mp, which):
    orig = ED.ghost_characteristic

    def bad(qm, n, gas):
        g = gas.gamma
        rho = qm[..., 0]
        u = qm[..., 1:4] / rho[..., None]
        p = ED.pressure(qm, g)
        c = np.sqrt(g * p / rho)
        un = np.sum(u * n, axis=-1)
        un_inf = np.sum(gas.u0 * n, axis=-1)
        Rp = un + 2.0 * c / (g - 1.0)
        Rm = un_inf + (1.0 if which == "Rm_sign" else -1.0) * 2.0 * gas.c0 / (g - 1.0)
        unb = 0.5 * (Rp + Rm)
        cb = (0.5 if which == "cb" else 0.25) * (g - 1.0) * (Rp - Rm)
        out = unb >= 0.0
        if which == "out_flipped":
            out = ~out
        s = np.where(out, p / rho ** g, gas.p0 / gas.rho0 ** g)
        if which == "entropy_inside":
            s = p / rho ** g
        ut = np.where(out[..., None], u - un[..., None] * n, gas.u0 - un_inf[..., None] * n)
        if which == "tangent_outside":
            ut = np.broadcast_to(gas.u0 - un_inf[..., None] * n, ut.shape)
        rhob = (cb * cb / (g * s)) ** (1.0 / (g - 1.0))
        ub = ut + unb[..., None] * n
        qp = np.empty_like(qm)
        qp[..., 0] = rhob
        qp[..., 1:4] = rhob[..., None] * ub
        qp[..., 4] = rhob * cb * cb / g / (g - 1.0) + 0.5 * rhob * np.sum(ub * ub, axis=-1)
        return qp
    _replace(mp, orig, bad)


def _inflow(mp, which):
    orig = ED.ghost_inflow

    def bad(qm, n, gas, t, amplitude, alpha):
        p = ED.inflow_pressure(t, gas, amplitude, alpha)
        rho = gas.rho0 * (p / gas.p0) ** (1.0 if which == "isothermal" else 1.0 / gas.gamma)
        un = (p - gas.p0) / (gas.rho0 * gas.c0)
        q = np.zeros(qm.shape)
        q[..., 0] = rho
        q[..., 1:4] = (1.0 if which == "outward" else -1.0) * np.asarray(rho * un)[..., None] * n
        q[..., 4] = p / (gas.gamma - 1.0) + 0.5 * rho * un * un
        return q
    _replace(mp, orig, bad)


def _inflow_two_pulses(mp):
    orig = ED.inflow_pressure

    def bad(t, gas, amplitude, alpha):
        t = np.asarray(t, dtype=np.float64)
        on = (t >= 0.0) & (t < 4.0 * np.pi / alpha)
        return gas.p0 * (1.0 + np.where(on, amplitude * (1.0 - np.cos(alpha * t)), 0.0))
    _replace(mp, orig, bad)


def _reference(mp, which):
    def post(s):
        if which == "Dr_transposed":
            s.Dr = s.Dr.T.copy()
        elif which == "Ds_Dt_swapped":
            s.Ds, s.Dt = s.Dt, s.Ds
        elif which == "lift_scaled":
            s.LIFT = 1.01 * s.LIFT
        elif which == "mass_scaled":
            s.M = 1.01 * s.M
        elif which == "face_mass_scaled":
            s.face_mass = [1.01 * fm for fm in s.face_mass]
        elif which == "fmask_swapped":
            F = s.Fmask.copy()
            F[[0, 1]] = F[[1, 0]]
            s.Fmask = F
    _after_init(mp, RE.ReferenceElement, post)


def _geometry(mp, which):
    def post(g):
        if which == "metric_transposed":
            g.drdx = np.transpose(g.drdx, (0, 2, 1)).copy()
        elif which == "normals_inward":
            g.nrm = -g.nrm
        elif which == "fscale_without_J":
            g.Fscale = g.sJ.copy()
        elif which == "sJ_is_area":
            g.sJ = g.area.copy()
            g.Fscale = g.sJ / g.J[:, None]
        elif which == "pairing_reversed":
            vp = g.vmapP.copy()
            inner = ~g.boundary
            vp[inner] = vp[inner][:, ::-1]
            g.vmapP = vp
    _after_init(mp, GE.Geometry, post)


def _surface_sign(mp):
    orig = ED.Solver._rhs

    def bad(self, q, psi, t, parts=False):
        saved = self.ref.LIFT
        self.ref.LIFT = -saved
        try:
            return orig(self, q, psi, t, parts)
        finally:
            self.ref.LIFT = saved
    mp.setattr(ED.Solver, "_rhs", bad)


def _totals_without_J(mp):
    mp.setattr(ED.Solver, "totals", lambda self, q: np.einsum("ij,kvj->v", self.ref.M, q))


def _ledger_weights_doubled(mp):
    _after_init(mp, ED.Solver, lambda s: setattr(s, "face_w", 2.0 * s.face_w))


def _lsrk(mp, which):
    if which == "B":
        b = list(ED.LSRK_B)
        b[2] = b[2] * 1.001
        mp.setattr(ED, "LSRK_B", b)
    else:
        c = list(ED.LSRK_C)
        mp.setattr(ED, "LSRK_C", [c[0]] + c[:-1])


def _lsrk_update_order(mp):
    def bad(self, q, t, dt, res=None, ledger=None):
        res = np.zeros_like(q) if res is None else res
        L_, Lres = (np.zeros(5), np.zeros(5)) if ledger is None else ledger
        psi, pres = self.psi, self.psi_res
        for k in range(5):
            a, b, c = float(ED.LSRK_A[k]), float(ED.LSRK_B[k]), float(ED.LSRK_C[k])
            rhs, lrhs, prhs = self.rhs_full(q, t + c * dt, psi)
            q = q + b * res                     # uses the previous stage's residual
            res = a * res + dt * rhs
            Lres = a * Lres + dt * lrhs
            L_ = L_ + b * Lres
            pres = a * pres + dt * prhs
            psi = psi + b * pres
        self.psi, self.psi_res = psi, pres
        return q, t + dt, res, (L_, Lres)
    mp.setattr(ED.Solver, "step", bad)


def _probe_coordinates_swapped(mp):
    orig = RE.ReferenceElement.interp_row
    mp.setattr(RE.ReferenceElement, "interp_row", lambda self, r, s, t: orig(self, s, r, t))


def _modal_rule_low(mp, which):
    orig = MD.tet_rule if which == "volume" else MD.tri_rule
    _replace(mp, orig, lambda degree: orig(max(degree - 1, 0)))


def _modal_face_own_rule(mp):
    """Each element integrates every face with its own rule, so the two sides
    of a face use different point sets where the rule's orientations differ."""
    def post(S):
        g, p = S.g, S.ref.p
        u, v, _ = MD.tri_rule(2 * p + 1)
        fpts = np.stack([MD.face_points(f, u, v) for f in range(4)])

        def phi(pts):
            flat = pts.reshape(-1, 3)
            out = RE.vandermonde3(p, flat[:, 0], flat[:, 1], flat[:, 2]) @ S.T
            return out.reshape(pts.shape[:-1] + (out.shape[1],))
        v1 = g.x[:, 0, :]
        Jm = np.linalg.inv(g.drdx)
        X = v1[:, None, None, :] + np.einsum("kij,fqj->kfqi", Jm, fpts + 1.0)
        verts = v1[:, None, :] + np.einsum("kij,cj->kci", Jm, MD.REF_VERTS + 1.0)
        fc = np.stack([verts[:, list(MD.FACE_VERTS[f])].mean(axis=1) for f in range(4)], axis=1)
        shift = fc - fc[g.EToE, g.EToF]
        r_nbr = -1.0 + np.einsum("kfij,kfqj->kfqi", g.drdx[g.EToE],
                                 X - shift[:, :, None, :] - v1[g.EToE][:, :, None, :])
        S.Phi_own = np.broadcast_to(phi(fpts)[None], X.shape[:3] + (S.T.shape[1],)).copy()
        S.Phi_nbr = phi(r_nbr)
    _after_init(mp, MD.ModalSolver, post)


def _modal_heun_wrong(mp):
    def bad(self, c, t, dt, ledger):
        k1, b1 = self.rhs(c, t)
        k2, b2 = self.rhs(c + dt * k1, t + dt)
        return c + dt * k2, ledger + 0.5 * dt * (b1 + b2)
    mp.setattr(MD.ModalSolver, "step", bad)


def _modal_ledger_half(mp):
    orig = MD.ModalSolver.rhs

    def bad(self, c, t=0.0):
        dc, led = orig(self, c, t)
        return dc, 0.5 * led
    mp.setattr(MD.ModalSolver, "rhs", bad)


def _modal_basis_scaled(mp):
    orig = MD.orthonormal_coefficients

    def bad(p):
        T = orig(p).copy()
        T[:, -1] *= 1.01
        return T
    _replace(mp, orig, bad)


def _mlp_missing_tanh_derivative(mp):
    def bad(w, X, T):
        X, T = np.asarray(X, dtype=np.float64), np.asarray(T, dtype=np.float64)
        p = ML.unpack(w)
        N = X.shape[0]
        y, (h1, h2) = ML.forward(w, X)
        d = y - T
        dy = 2.0 * d / N
        g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
        dz2 = dy @ p["W3"].T                      # (1 - h2^2) dropped
        g["W2"], g["b2"] = h1.T @ dz2, dz2.sum(axis=0)
        dz1 = (dz2 @ p["W2"].T) * (1.0 - h1 * h1)
        g["W1"], g["b1"] = X.T @ dz1, dz1.sum(axis=0)
        return np.sum(d * d) / N, ML.pack(g)
    _replace(mp, ML.loss_and_grad, bad)


def _mlp_loss_summed(mp):
    orig = ML.loss_and_grad

    def bad(w, X, T):
        loss, g = orig(w, X, T)
        N = np.asarray(X).shape[0]
        return loss * N, g * N
    _replace(mp, orig, bad)


def _adam_without_bias_correction(mp):
    def bad(w, X, T, iters, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        w = np.array(w, dtype=np.float64)
        m, v, hist = np.zeros_like(w), np.zeros_like(w), []
        for _ in range(iters):
            loss, g = ML.loss_and_grad(w, X, T)
            hist.append(loss)
            m = beta1 * m + (1 - beta1) * g
            v = beta2 * v + (1 - beta2) * g * g
            w = w - lr * m / (np.sqrt(v) + eps)
        return w, np.array(hist)
    _replace(mp, ML.adam, bad)


def _features_wout_sign(mp):
    orig = ML.features

    def bad(qp, n, x, psi, gas, radius):
        f, s = orig(qp, n, x, psi, gas, radius)
        rho = gas.rho0 + qp[..., 0]
        un = np.sum(qp[..., 1:4] / rho[..., None] * n, axis=-1)
        f = f.copy()
        f[..., 0] -= 2.0 * un / (gas.c0 * s)      # p' - rho0 c0 u.n instead of +
        return f, s
    _replace(mp, orig, bad)


def _probe_tie_last(mp):
    orig = ED.Probes.__init__

    def init(self, geom, pts, tol=1e-12):
        orig(self, geom, pts, tol)
        pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
        v = geom.verts
        T = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
        for i, x in enumerate(pts):
            lam = np.linalg.solve(T, (x - v[:, 0])[:, :, None])[:, :, 0]
            hit = np.nonzero((lam.min(axis=1) >= -tol) & (1.0 - lam.sum(axis=1) >= -tol))[0]
            e = hit[-1]                               # the last element, not the first
            r, s, t = -1 + 2 * lam[e]
            self.elem[i] = e
            self.rows[i] = geom.ref.interp_row(r, s, t)[0]
    mp.setattr(ED.Probes, "__init__", init)


def _invariants_swapped(mp):
    orig = ED.acoustic_invariants

    def bad(qp, n, gas):
        wout, win = orig(qp, n, gas)
        return win, wout
    _replace(mp, orig, bad)


def _memory(mp, which):
    def bad(psi, wout, r, gas):
        if which == "sign":
            return -(gas.c0 / (2.0 * r)) * (psi - wout)
        return -(gas.c0 / r) * (psi + wout)
    _replace(mp, ED.memory_rate, bad)


def _learned_ghost(mp, which):
    orig = ED.ghost_learned

    def bad(qm, n, x, psi, gas, w, radius):
        q0 = gas.freestream()
        qc = ED.ghost_characteristic(qm, n, gas)
        feats, s = ML.features(qm - q0, n, x, psi, gas, radius)
        y, _ = ML.forward(w, feats.reshape(-1, ML.N_IN))
        y = y.reshape(qm.shape)
        _, wi_c = ED.acoustic_invariants(qc - q0, n, gas)
        pref = gas.rho0 * gas.c0 ** 2
        g = psi + pref * s * y[..., 0]
        if which != "unbounded":
            lim = np.maximum(np.abs(wi_c), pref * s)
            g = np.clip(g, -lim, lim)
        D = g - wi_c
        c0 = gas.c0
        q = qc.copy()
        q[..., 0] += D / (2 * c0 * c0)
        q[..., 1:4] += (1.0 if which == "momentum_sign" else -1.0) * (D / (2 * c0))[..., None] * n
        q[..., 4] += D / (2 * (gas.gamma - 1.0))
        return q
    _replace(mp, orig, bad)


def _stable_dt_linear_in_order(mp):
    def bad(self, q, cfl=0.5):
        qn = np.transpose(q, (0, 2, 1))
        rho = qn[..., 0]
        u = qn[..., 1:4] / rho[..., None]
        c = np.sqrt(self.gas.gamma * ED.pressure(qn, self.gas.gamma) / rho)
        smax = np.max(np.linalg.norm(u, axis=-1) + c)
        return cfl * np.min(GE.inscribed_radius(self.g)) / ((self.ref.p + 1) * smax)
    mp.setattr(ED.Solver, "stable_dt", bad)


P = functools.partial
MISTAKES = {
    "Eq. 1 fluxes as printed": (_flux_as_printed, [E.test_flux_jacobian_eigenvalues]),
    "pressure with gamma for gamma - 1": (P(_pressure_factor, which="gamma"),
                                          [E.test_eq3_scaled_free_stream]),
    "pressure without the 1/2": (P(_pressure_factor, which="half"),
                                 [E.test_flux_jacobian_eigenvalues]),
    "LLF dissipation sign": (P(_llf, which="sign"), [E.test_inflow_ghost_injects_the_planar_wave]),
    "LLF with the smaller wave speed": (P(_llf, which="min"),
                                        [E.test_llf_dissipation_is_the_larger_spectral_radius]),
    "central flux": (P(_llf, which="central"),
                     [E.test_llf_dissipation_is_the_larger_spectral_radius]),
    "wave speed without |.|": (_wave_speed_signed, [E.test_llf_consistency_and_antisymmetry]),
    "slip wall removes the normal velocity only": (
        _slip_wall_half, [E.test_slip_wall_flux_has_no_mass_or_energy_flux]),
    "characteristic c_b factor": (P(_characteristic, which="cb"),
                                  [E.test_characteristic_ghost_free_stream_and_outgoing_wave]),
    "characteristic R- sign": (P(_characteristic, which="Rm_sign"),
                               [E.test_characteristic_ghost_free_stream_and_outgoing_wave]),
    "characteristic inflow/outflow switched": (
        P(_characteristic, which="out_flipped"),
        [E.test_characteristic_ghost_free_stream_and_outgoing_wave]),
    "characteristic entropy always from inside": (
        P(_characteristic, which="entropy_inside"),
        [E.test_characteristic_ghost_free_stream_and_outgoing_wave]),
    "characteristic tangential velocity always from outside": (
        P(_characteristic, which="tangent_outside"),
        [E.test_characteristic_ghost_passes_an_outgoing_shear_wave]),
    "inflow velocity along the outward normal": (
        P(_inflow, which="outward"), [E.test_inflow_ghost_injects_the_planar_wave]),
    "inflow density isothermal": (P(_inflow, which="isothermal"),
                                  [E.test_inflow_ghost_injects_the_planar_wave]),
    "inflow pulse repeated": (_inflow_two_pulses,
                              [E.test_inflow_ghost_is_the_free_stream_outside_the_pulse]),
    "Dr transposed": (P(_reference, which="Dr_transposed"),
                      [P(R.test_derivative_matrices_exact_on_polynomials, 2)]),
    "Ds and Dt swapped": (P(_reference, which="Ds_Dt_swapped"),
                          [P(R.test_derivative_matrices_exact_on_polynomials, 2)]),
    "LIFT scaled": (P(_reference, which="lift_scaled"), [P(R.test_face_mass_and_lift, 2)]),
    "mass matrix scaled": (P(_reference, which="mass_scaled"),
                           [P(R.test_mass_matrix_against_quadrature, 2)]),
    "face mass scaled": (P(_reference, which="face_mass_scaled"), [P(R.test_face_mass_and_lift, 2)]),
    "face node lists of two faces swapped": (P(_reference, which="fmask_swapped"),
                                             [P(R.test_face_mass_and_lift, 2)]),
    "metric transposed": (P(_geometry, which="metric_transposed"),
                          [E.test_strong_form_equals_weak_form_quadrature]),
    "normals inward": (P(_geometry, which="normals_inward"),
                       [E.test_strong_form_equals_weak_form_quadrature]),
    "Fscale without 1/J": (P(_geometry, which="fscale_without_J"),
                           [E.test_strong_form_equals_weak_form_quadrature]),
    "surface Jacobian = area": (P(_geometry, which="sJ_is_area"),
                                [E.test_strong_form_equals_weak_form_quadrature]),
    "face nodes paired in reverse": (P(_geometry, which="pairing_reversed"),
                                     [E.test_rhs_does_not_depend_on_the_vertex_order]),
    "surface term sign": (_surface_sign, [E.test_strong_form_equals_weak_form_quadrature]),
    "totals without J": (_totals_without_J, [E.test_discrete_conservation_periodic_and_ledger]),
    "ledger weights doubled": (_ledger_weights_doubled,
                               [E.test_discrete_conservation_periodic_and_ledger]),
    "Runge-Kutta B coefficient": (P(_lsrk, which="B"), [E.test_lsrk_coefficients_and_order_conditions]),
    "Runge-Kutta stage times shifted": (P(_lsrk, which="C"),
                                        [E.test_lsrk_coefficients_and_order_conditions]),
    "Runge-Kutta update order": (_lsrk_update_order, [E.test_discrete_conservation_periodic_and_ledger]),
    "probe coordinates swapped": (_probe_coordinates_swapped, [E.test_probes_interpolate_linear_fields]),
    "time step with (p+1) for (p+1)^2": (_stable_dt_linear_in_order,
                                         [E.test_stable_dt_closed_form_on_the_lattice]),
    "probe on a shared point takes the last element": (_probe_tie_last,
                                                       [E.test_probes_interpolate_linear_fields]),
    "acoustic invariants swapped": (_invariants_swapped, [L.test_learned_target_is_the_incoming_invariant_gap]),
    "memory driven by -w_out": (P(_memory, which="sign"),
                                [L.test_memory_reproduces_the_spherical_incoming_invariant]),
    "memory rate c0/r": (P(_memory, which="rate"),
                         [L.test_memory_reproduces_the_spherical_incoming_invariant]),
    "learned ghost momentum increment sign": (
        P(_learned_ghost, which="momentum_sign"),
        [L.test_learned_ghost_moves_only_the_incoming_invariant_within_the_bound]),
    "learned ghost unbounded": (
        P(_learned_ghost, which="unbounded"),
        [L.test_learned_ghost_moves_only_the_incoming_invariant_within_the_bound]),
    "modal volume rule one degree short": (P(_modal_rule_low, which="volume"),
                                           [P(M.test_rules_integrate_monomials_exactly, 4)]),
    "modal face rule one degree short": (P(_modal_rule_low, which="face"),
                                         [P(M.test_rules_integrate_monomials_exactly, 4)]),
    "modal faces integrated on each side's own points": (
        _modal_face_own_rule, [M.test_discrete_conservation_periodic_and_ledger]),
    "Heun's second stage": (_modal_heun_wrong, [M.test_heun_amplification_on_a_linear_problem]),
    "modal ledger halved": (_modal_ledger_half, [M.test_discrete_conservation_periodic_and_ledger]),
    "modal basis not orthonormal": (_modal_basis_scaled, [P(M.test_basis_is_orthonormal, 2)]),
    "backprop without a tanh derivative": (_mlp_missing_tanh_derivative,
                                           [L.test_gradient_against_central_differences]),
    "loss summed, not averaged": (_mlp_loss_summed, [L.test_zero_weights_closed_form]),
    "Adam without bias correction": (_adam_without_bias_correction, [L.test_first_adam_step_moves_by_lr]),
    "outgoing invariant with the wrong sign": (_features_wout_sign, [L.test_features_definition]),
}


@pytest.mark.parametrize("name", list(MISTAKES))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    plant, pins = MISTAKES[name]
    plant(monkeypatch)
    caught = 0
    with np.errstate(all="ignore"):
        for pin in pins:
            try:
                pin()
            except AssertionError:
                caught += 1
    assert caught > 0, f"no pin caught: {name}"
