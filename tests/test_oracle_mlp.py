"""Pins of the oracle's network and learned closure (CPU)."""
import numpy as np
import pytest

from oracle import mlp
from oracle.euler_dg import Gas, ghost_characteristic, ghost_learned


def test_parameter_count_and_packing():
    assert mlp.N_PARAMS == 12 * 64 + 64 + 64 * 64 + 64 + 64 * 5 + 5 == 5317
    w = np.arange(mlp.N_PARAMS, dtype=np.float64)
    p = mlp.unpack(w)
    assert p["W1"][0, 1] == 1 and p["b1"][0] == 768 and p["b3"][-1] == mlp.N_PARAMS - 1
    np.testing.assert_array_equal(mlp.pack(p), w)


def test_gradient_against_central_differences():
    rng = np.random.default_rng(0)
    w = mlp.init_params(seed=1)
    w += 0.1 * rng.normal(size=w.shape)           # nonzero biases too
    X = rng.normal(size=(40, 12))
    T = rng.normal(size=(40, 5))
    loss, g = mlp.loss_and_grad(w, X, T)
    idx = rng.choice(mlp.N_PARAMS, 300, replace=False)
    idx = np.concatenate([idx, np.arange(mlp.N_PARAMS - 5, mlp.N_PARAMS)])
    for i in idx:
        h = 1e-6
        e = np.zeros_like(w)
        e[i] = h
        fd = (mlp.loss_and_grad(w + e, X, T)[0] - mlp.loss_and_grad(w - e, X, T)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9)


def test_zero_weights_closed_form():
    rng = np.random.default_rng(2)
    w = np.zeros(mlp.N_PARAMS)
    b3 = rng.normal(size=5)
    w[-5:] = b3
    X = rng.normal(size=(10, 12))
    T = rng.normal(size=(10, 5))
    y, _ = mlp.forward(w, X)
    np.testing.assert_array_equal(y, np.tile(b3, (10, 1)))
    loss, g = mlp.loss_and_grad(w, X, T)
    assert loss == pytest.approx(np.sum((b3 - T) ** 2) / 10)
    np.testing.assert_allclose(g[-5:], 2 * np.mean(b3 - T, axis=0))
    # with W3 = 0 nothing reaches the first layers
    assert np.all(g[:-5 - 64 * 5] == 0)


def test_first_adam_step_moves_by_lr():
    rng = np.random.default_rng(3)
    w0 = mlp.init_params(seed=4)
    X = rng.normal(size=(20, 12))
    T = rng.normal(size=(20, 5))
    _, g = mlp.loss_and_grad(w0, X, T)
    w1, hist = mlp.adam(w0, X, T, iters=1, lr=1e-3)
    # bias-corrected first moment / root second moment = g / (|g| + eps)
    nz = np.abs(g) > 1e-6
    np.testing.assert_allclose((w0 - w1)[nz], 1e-3 * g[nz] / (np.abs(g[nz]) + 1e-8), rtol=1e-9)
    w50, hist = mlp.adam(w0, X, T, iters=50, lr=1e-2)
    assert hist[-1] < 0.5 * hist[0]


def _trace_states(gas, rng, k=7, amp=1e-3):
    n = rng.normal(size=(k, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    qm = np.tile(gas.freestream(), (k, 1))
    qm[:, 0] *= 1 + amp * rng.normal(size=k)
    qm[:, 1:4] = amp * gas.rho0 * gas.c0 * rng.normal(size=(k, 3))
    qm[:, 4] *= 1 + amp * rng.normal(size=k)
    psi = amp * gas.rho0 * gas.c0 ** 2 * rng.normal(size=k)
    return qm, n, rng.normal(size=(k, 3)), psi


def test_learned_ghost_with_zero_output_is_the_spherical_condition():
    """A network whose output is zero leaves the characteristic ghost's
    outgoing invariant alone and sets its incoming invariant to the memory
    psi (linearised invariants: to second order in the amplitude); with
    psi = 0 as well it is the characteristic ghost moved to w_in = 0."""
    from oracle.euler_dg import acoustic_invariants
    gas = Gas(1.4, 1.225, 101325.0)
    qm, n, x, psi = _trace_states(gas, np.random.default_rng(5))
    q0 = gas.freestream()
    gc = ghost_characteristic(qm, n, gas)
    w = np.zeros(mlp.N_PARAMS)
    gl = ghost_learned(qm, n, x, psi, gas, w, 1.0)
    wo_c, wi_c = acoustic_invariants(gc - q0, n, gas)
    wo_l, wi_l = acoustic_invariants(gl - q0, n, gas)
    wo_m, _ = acoustic_invariants(qm - q0, n, gas)
    amp = np.abs(wo_m) + np.abs(psi)
    tol = 1e-2 * (amp + np.abs(psi - wi_c))
    assert np.all(np.abs(wi_l - psi) <= tol)
    assert np.all(np.abs(wo_l - wo_c) <= tol)
    # exactly: the increment is D = psi - w_in,c along the incoming wave
    D = psi - wi_c
    want = gc.copy()
    want[:, 0] += D / (2 * gas.c0 ** 2)
    want[:, 1:4] -= (D / (2 * gas.c0))[:, None] * n
    want[:, 4] += D / (2 * (gas.gamma - 1.0))
    np.testing.assert_allclose(gl, want, rtol=1e-15, atol=0)


def test_learned_ghost_moves_only_the_incoming_invariant_within_the_bound():
    from oracle.euler_dg import acoustic_invariants
    gas = Gas(1.4, 1.225, 101325.0)
    rng = np.random.default_rng(6)
    qm, n, x, psi = _trace_states(gas, rng, k=50)
    q0 = gas.freestream()
    gc = ghost_characteristic(qm, n, gas)
    wo_m, _ = acoustic_invariants(qm - q0, n, gas)
    wo_c, wi_c = acoustic_invariants(gc - q0, n, gas)
    _, s = mlp.features(qm - q0, n, x, psi, gas, 1.0)
    pref = gas.rho0 * gas.c0 ** 2
    # the bound is |w_out| + |psi| (or the characteristic ghost's own |w_in|)
    np.testing.assert_allclose(pref * s, np.abs(wo_m) + np.abs(psi) + pref * 1e-12, rtol=1e-12)
    amp = np.abs(wo_m) + np.abs(psi)
    for b0 in (0.05, -0.05, 1e3):              # small corrections, and a huge one (clipped)
        w = np.zeros(mlp.N_PARAMS)
        w[-5] = b0                             # constant output 0 = b0
        gl = ghost_learned(qm, n, x, psi, gas, w, 1.0)
        wo_l, wi_l = acoustic_invariants(gl - q0, n, gas)
        lim = np.maximum(np.abs(wi_c), pref * s)
        want = np.clip(psi + pref * s * b0, -lim, lim)
        # outgoing invariant unchanged, incoming one moved to the bounded target
        # (linearised invariants: second-order terms ~ amplitude x change)
        tol = 1e-2 * (amp + np.abs(want - wi_c))
        assert np.all(np.abs(wo_l - wo_c) <= tol)
        assert np.all(np.abs(wi_l - want) <= tol)
    # the huge correction saturates at the bound
    assert np.all(np.abs(np.abs(wi_l) - lim) <= 1e-2 * (amp + lim))


def test_learned_target_is_the_incoming_invariant_gap():
    """The target is what the outer trace's incoming invariant adds to the
    memory psi, in units of rho0 c0^2 s; it vanishes where the outer trace
    carries exactly psi."""
    from oracle.euler_dg import acoustic_invariants, learned_target
    gas = Gas(1.4, 1.225, 101325.0)
    rng = np.random.default_rng(8)
    qm, n, _, psi = _trace_states(gas, rng, k=20)
    qo, _, _, _ = _trace_states(gas, rng, k=20)
    q0 = gas.freestream()
    y = learned_target(qm, qo, n, psi, gas)
    _, wi_o = acoustic_invariants(qo - q0, n, gas)
    wo_m, _ = acoustic_invariants(qm - q0, n, gas)
    s = (np.abs(wo_m) + np.abs(psi)) / (gas.rho0 * gas.c0 ** 2) + 1e-12
    np.testing.assert_allclose(y[:, 0] * gas.rho0 * gas.c0 ** 2 * s, wi_o - psi, rtol=1e-12)
    assert np.all(y[:, 1:] == 0)
    # an outer trace whose incoming invariant is psi: nothing to learn. Move
    # qo along the incoming wave (isentropic increments) until w_in = psi.
    qo2 = qo.copy()
    for _ in range(30):                         # the invariants are nonlinear: iterate
        _, wi = acoustic_invariants(qo2 - q0, n, gas)
        D = psi - wi
        qo2[:, 0] += D / (2 * gas.c0 ** 2)
        qo2[:, 1:4] -= (D / (2 * gas.c0))[:, None] * n
        qo2[:, 4] += D / (2 * (gas.gamma - 1.0))
    assert np.allclose(learned_target(qm, qo2, n, psi, gas)[:, 0], 0, atol=1e-9)


def test_features_definition():
    gas = Gas(1.4, 1.0, 1.0 / 1.4)            # c0 = 1, p0 = 1/1.4, rho0 c0^2 = 1
    q = np.array([[0.01, 0.02, -0.03, 0.04, 0.05]])
    n = np.array([[0.0, 0.0, 1.0]])
    x = np.array([[0.5, 0.0, 0.0]])
    psi = np.array([-0.007])
    f, s = mlp.features(q, n, x, psi, gas, 2.0)
    rho = 1.01
    pp = 0.4 * (0.05 - 0.5 * (0.02 ** 2 + 0.03 ** 2 + 0.04 ** 2) / rho)
    wout = pp + 0.04 / rho
    assert s[0] == pytest.approx(abs(wout) + 0.007 + 1e-12)
    assert f[0, 0] == pytest.approx(wout / s[0])
    assert f[0, 1] == pytest.approx((0.01 - pp) / s[0])
    np.testing.assert_allclose(f[0, 2:5], [0.02 / rho / s[0], -0.03 / rho / s[0], 0.0], atol=1e-15)
    np.testing.assert_allclose(f[0, 5:8], [0, 0, 1])
    np.testing.assert_allclose(f[0, 8:11], [0.25, 0, 0])
    assert f[0, 11] == pytest.approx(-0.007 / s[0])
    assert abs(f[0, 0]) + abs(f[0, 11]) == pytest.approx(1.0)
    # the incoming invariant of the trace does not enter the features
    q2 = q.copy()
    dwin = 1e-3                                # change p' by dwin/2 and rho0 c0 u_n by -dwin/2
    q2[0, 4] += dwin / 2 / 0.4
    q2[0, 3] -= dwin / 2
    f2, s2 = mlp.features(q2, n, x, psi, gas, 2.0)
    assert abs(s2[0] - s[0]) < 2e-2 * dwin          # second order: amplitude x change


def test_memory_reproduces_the_spherical_incoming_invariant():
    """Closed form: an outgoing spherical wave p = f(t - r/c0)/r of linear
    acoustics has, at radius r, w_out = 2 f/r + c0 F/r^2 and
    w_in = -c0 F/r^2 (F the time integral of f, from the radial momentum
    equation). Driving the memory with that w_out, integrated by the
    scheme's own Runge-Kutta stages, reproduces w_in."""
    from scipy.special import erf
    from oracle.euler_dg import LSRK_A, LSRK_B, LSRK_C, memory_rate
    gas = Gas(1.4, 1.225, 101325.0)
    c0 = gas.c0
    for r, sig in ((1.0, 0.3 / c0), (2.5, 0.1 / c0)):
        def f(tau):
            return 50.0 * np.exp(-(tau / sig) ** 2)

        def F(tau):
            return 50.0 * sig * np.sqrt(np.pi) / 2 * (1.0 + erf(tau / sig))

        def wout(t):
            return 2 * f(t - r / c0) / r + c0 * F(t - r / c0) / r ** 2

        t, dt = r / c0 - 6 * sig, sig / 40
        psi, res = 0.0, 0.0
        err, peak = 0.0, 0.0
        for _ in range(600):
            for a, b, c in zip(LSRK_A, LSRK_B, LSRK_C):
                res = float(a) * res + dt * memory_rate(psi, wout(t + float(c) * dt), r, gas)
                psi = psi + float(b) * res
            t += dt
            exact = -c0 * F(t - r / c0) / r ** 2
            err = max(err, abs(psi - exact))
            peak = max(peak, abs(exact))
        assert err <= 1e-6 * peak, (r, err, peak)
        # and the characteristic ghost's w_in = 0 misses all of it: a few per
        # cent (narrow pulse far out) to a quarter of the outgoing peak 100/r
        assert peak > 0.03 * 100.0 / r


def test_solver_memory_decays_on_the_free_stream():
    """On the free stream w_out = 0, so a memory decays as
    psi0 exp(-c0 t / 2r). Trace faces (whose memory feeds nothing back) start
    from random memories and decay so; learned faces start from zero, so the
    zero network (the spherical condition, w_in = psi = 0) keeps the free
    stream and their memories stay zero."""
    from oracle.euler_dg import LEARNED, Solver
    from oracle.geometry import Geometry
    from oracle.reference_element import ReferenceElement
    from paper_1710_03887_gb300 import workloads as W
    gas = Gas(1.4, 1.225, 101325.0)
    xyz, EToV = W.kuhn_cube(2, jitter=0.1, seed=1)
    geom = Geometry(ReferenceElement(1), xyz, EToV)
    S = Solver(geom, gas, bc_mode={0: LEARNED}, mlp=(np.zeros(mlp.N_PARAMS), 0.7))
    # interior faces away from the origin (where r is floored)
    inner = np.nonzero(~geom.boundary)
    fx = geom.x[inner[0][:, None], geom.ref.Fmask[inner[1]]]
    far = np.nonzero(np.linalg.norm(fx, axis=-1).min(axis=1) > 0.2)[0][:5]
    S.set_trace_faces(inner[0][far], inner[1][far])
    nl = S.n_learned
    assert nl == int(geom.boundary.sum()) and len(S.mem_elem) == nl + 5
    rng = np.random.default_rng(3)
    psi0 = rng.normal(size=S.psi.shape) * 100.0
    psi0[:nl] = 0.0
    S.psi = psi0.copy()
    q = W.uniform_state(geom.K, geom.ref.Np, gas.rho0, (0, 0, 0), gas.p0, gas.gamma)
    q0 = q.copy()
    dt = 1e-4
    res, led, t = None, None, 0.0
    for _ in range(20):
        q, t, res, led = S.step(q, t, dt, res, led)
    np.testing.assert_allclose(q, q0, rtol=1e-14, atol=1e-9)
    r = np.linalg.norm(S.mem_x, axis=-1)
    np.testing.assert_allclose(S.psi, psi0 * np.exp(-gas.c0 * t / (2 * r)), rtol=1e-9)
    assert np.all(S.psi[:nl] == 0.0) and np.all(np.abs(S.psi[nl:]) > 0)


def test_spherical_weights_realise_the_memory_condition():
    """The spherical-wave parameter set is the all-zero network: every output
    is zero, so the closure's incoming invariant is the memory psi."""
    from paper_1710_03887_gb300 import learned_bc as L
    w = L.spherical_weights().astype(np.float64)
    X = np.random.default_rng(4).uniform(-1, 1, size=(500, mlp.N_IN))
    y, _ = mlp.forward(w, X)
    assert np.all(y == 0)


def test_header_worked_example_matches_features():
    """The boundary header documents the closure's features with a worked
    example (EXAMPLE_FEATURES); the oracle's feature definition gives those
    numbers for that trace, so the header's contract is the one computed."""
    import re
    from pathlib import Path
    text = (Path(__file__).resolve().parent.parent / "include" / "dg_euler.h").read_text()
    m = re.search(r"EXAMPLE_FEATURES:([-0-9.\s]+)", text)
    want = np.array([float(v) for v in m.group(1).split()])
    assert want.size == mlp.N_IN
    gas = Gas(1.4, 1.0, 1.0 / 1.4)              # rho0 = 1, c0 = 1
    q = np.array([[0.01, 0.02, -0.03, 0.04, 0.05]])
    n = np.array([[0.0, 0.0, 1.0]])
    x = np.array([[0.3, -0.4, 1.2]])
    f, s = mlp.features(q, n, x, np.array([-0.02]), gas, 2.0)
    np.testing.assert_allclose(f[0], want, rtol=0, atol=1e-10)
    m = re.search(r"s = ([0-9.]+) \(\+1e-12\)", text)
    assert s[0] == pytest.approx(float(m.group(1)) + 1e-12, abs=1e-10)
    # the same vector by hand from the header's definitions
    rho = 1.01
    u = q[0, 1:4] / rho
    pp = 0.4 * (0.05 - 0.5 * np.sum(q[0, 1:4] ** 2) / rho)
    wout = pp + u[2]
    amp = abs(wout) + 0.02 + 1e-12
    hand = np.concatenate([[wout / amp, (0.01 - pp) / amp], [u[0] / amp, u[1] / amp, 0.0],
                           [0, 0, 1], [0.15, -0.2, 0.6], [-0.02 / amp]])
    np.testing.assert_allclose(want, hand, rtol=0, atol=1e-10)
