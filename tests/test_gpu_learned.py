"""Learned boundary closure on the GPU: network kernels against the float64
oracle, trace sampling, the closure inside the operator, and the gain over
the characteristic condition it is meant to improve on.

Tolerances (float32 kernels against float64): a loss or a gradient entry is a
sum over samples of products of O(1) values, so 1e-4 of the largest entry;
forward outputs 1e-5; the right-hand side with the closure as in
test_gpu_f32 (2e-5 of max |rhs|).
"""
import numpy as np
import pytest

from oracle import mlp as OM
from oracle.euler_dg import LEARNED, Gas
from oracle.euler_dg import Solver as OSolver
from oracle.geometry import Geometry
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import learned_bc as L
from paper_1710_03887_gb300 import workloads as W

from ._cases import SI, rel_err

pytestmark = pytest.mark.gpu


def _weights(seed, out_scale=1.0):
    rng = np.random.default_rng(seed)
    w = OM.init_params(seed=seed) + 0.05 * rng.normal(size=OM.N_PARAMS)
    w[-5 - 64 * 5:] *= out_scale
    return w


def _solver():
    return B.Solver(2, precision=B.DG_PREC_F32, **SI)


def test_mlp_loss_gradient_and_forward_match_oracle(cuda_device):
    import torch
    rng = np.random.default_rng(0)
    N = 1000
    X = rng.normal(size=(N, 12)).astype(np.float32)
    Y = rng.normal(size=(N, 5)).astype(np.float32)
    w = _weights(1).astype(np.float32)
    S = _solver()
    S.set_bc_mlp(w, 1.0)
    dX = torch.from_numpy(X).to(cuda_device)
    dY = torch.from_numpy(Y).to(cuda_device)
    loss, grad = S.mlp_loss_grad(dX, dY)
    lo, go = OM.loss_and_grad(w.astype(np.float64), X, Y)
    assert loss == pytest.approx(lo, rel=1e-5)
    assert np.abs(grad - go).max() <= 1e-4 * np.abs(go).max()
    out = torch.empty((N, 5), dtype=torch.float32, device=cuda_device)
    S.mlp_forward(dX, out)
    yo, _ = OM.forward(w.astype(np.float64), X)
    assert np.abs(out.cpu().numpy() - yo).max() <= 1e-5 * np.abs(yo).max()
    # the gradient is deterministic
    loss2, grad2 = S.mlp_loss_grad(dX, dY)
    assert loss2 == loss and np.array_equal(grad, grad2)


def test_mlp_adam_training_matches_oracle(cuda_device):
    import torch
    rng = np.random.default_rng(2)
    N = 2000
    X = rng.normal(size=(N, 12)).astype(np.float32)
    Y = np.tanh(X[:, :5] * 0.7 + 0.2 * X[:, 5:10]).astype(np.float32)   # a learnable map
    w0 = OM.init_params(seed=3).astype(np.float32)
    S = _solver()
    S.set_bc_mlp(w0, 1.0)
    hist = S.mlp_train(torch.from_numpy(X).to(cuda_device), torch.from_numpy(Y).to(cuda_device),
                       60, 3e-3)
    _, ho = OM.adam(w0.astype(np.float64), X, Y, 60, 3e-3)
    np.testing.assert_allclose(hist[:10], ho[:10], rtol=1e-4)
    assert hist[-1] == pytest.approx(ho[-1], rel=2e-2)
    assert hist[-1] < 0.5 * hist[0]


@pytest.mark.parametrize("p,prec", [(2, B.DG_PREC_F32), (4, B.DG_PREC_F32),
                                    (4, B.DG_PREC_F32_TC)])
def test_learned_closure_rhs_matches_oracle(cuda_device, p, prec):
    """The closure inside one right-hand side, against the oracle's: p = 2,
    and p = 4 (15 nodes per face: the production configuration's order) in
    both float32 forms."""
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=4)
    gas = Gas(SI["gamma"], SI["rho0"], SI["p0"])
    ref = ReferenceElement(p)
    geom = Geometry(ref, xyz, EToV)
    w = _weights(5, out_scale=0.2)
    orc = OSolver(geom, gas, bc_mode={0: LEARNED}, mlp=(w, 1.3))
    q = W.random_smooth_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, seed=6)
    ro = orc.rhs(q)
    S = B.Solver(p, precision=prec, **SI)
    S.upload_mesh(xyz, EToV)
    S.set_bc(0, B.DG_BC_LEARNED)
    S.set_bc_mlp(w.astype(np.float32), 1.3)
    S.set_state(q)
    err = rel_err(S.eval_rhs(), ro)
    assert np.all(err < 2e-5), err
    # the correction matters: the characteristic condition gives a different rhs
    orc_c = OSolver(geom, gas)
    assert np.abs(orc_c.rhs(q) - ro).max() > 1e-3 * np.abs(ro).max()


@pytest.mark.parametrize("prec", [B.DG_PREC_F32, B.DG_PREC_F32_TC])
def test_learned_closure_run_matches_oracle(cuda_device, prec):
    """Twenty steps with the closure and its memory against the float64 oracle:
    the memory grows from zero with the outgoing waves and feeds the network."""
    p = 2
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=8)
    gas = Gas(SI["gamma"], SI["rho0"], SI["p0"])
    geom = Geometry(ReferenceElement(p), xyz, EToV)
    w = _weights(9, out_scale=0.2)
    w[11 * 64:12 * 64] *= 20.0                  # make the memory feature matter
    orc = OSolver(geom, gas, bc_mode={0: LEARNED}, mlp=(w, 1.0))
    q0 = W.gaussian_pulse_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.02, 0.3,
                                center=(0.2, -0.1, 0.1))
    dt = orc.stable_dt(q0, 0.5)
    qo, _, _, _ = orc.run(q0, dt, 20)
    assert np.abs(orc.psi).max() > 1e-3 * 0.02 * SI["p0"]      # the memory is in play
    S = B.Solver(p, precision=prec, **SI)
    S.upload_mesh(xyz, EToV)
    S.set_bc(0, B.DG_BC_LEARNED)
    S.set_bc_mlp(w.astype(np.float32), 1.0)
    S.set_state(q0)
    S.step(20, dt)
    qg, _ = S.get_state()
    base = W.uniform_state(geom.K, geom.ref.Np, SI["rho0"], (0, 0, 0), SI["p0"], SI["gamma"])
    num = np.abs(qg - qo).max(axis=(0, 2))
    den = np.abs(qo - base).max(axis=(0, 2))
    assert np.all(num <= 2e-4 * den), num / den
    # the same run with the characteristic condition ends elsewhere
    oc = OSolver(geom, gas)
    qc, _, _, _ = oc.run(q0, dt, 20)
    assert np.abs(qc - qo).max(axis=(0, 2))[4] > 1e-3 * den[4]     # 5x the tolerance


def test_trace_samples_match_oracle(cuda_device):
    import torch
    p = 2
    nested = L.nested_ball(8)
    S = B.Solver(p, precision=B.DG_PREC_F32, **SI)
    S.upload_mesh(*nested.big)
    elem, face = L.trace_faces(S, nested)
    assert len(elem) == 12 * 4 ** 2                 # the r = 1 sphere: 2 triangles per lattice square
    S.set_trace_faces(elem, face)
    geom = Geometry(ReferenceElement(p), *nested.big)
    gas = Gas(SI["gamma"], SI["rho0"], SI["p0"])
    q0 = W.gaussian_pulse_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, 0.3,
                                center=(0.3, 0.2, -0.1))
    orc = OSolver(geom, gas)
    orc.set_trace_faces(elem, face)
    dt = orc.stable_dt(q0, 0.5)
    steps = 40                                       # the pulse reaches r = 1
    qo, _, _, _ = orc.run(q0, dt, steps)
    fo, yo, so = orc.trace_samples(qo)
    S.set_state(q0)
    S.step(steps, dt)
    n = len(elem) * S.Nfp
    X = torch.empty((n, 12), dtype=torch.float32, device=cuda_device)
    Y = torch.empty((n, 5), dtype=torch.float32, device=cuda_device)
    amp = torch.empty((n,), dtype=torch.float32, device=cuda_device)
    S.sample_traces(X, Y, amp)
    S.sync()
    Xg, Yg, ag = X.cpu().numpy(), Y.cpu().numpy(), amp.cpu().numpy()
    fo, yo, so = fo.reshape(-1, 12), yo.reshape(-1, 5), so.reshape(-1)
    assert np.abs(orc.psi).max() > 1e-3 * 0.05 * SI["p0"]     # the memory has filled
    # compare where the wave has arrived (s above 1e-3 of its largest value):
    # features and targets are ratios by s, a float32 sum that partly cancels
    live = so > 1e-3 * so.max()
    assert live.mean() > 0.5
    np.testing.assert_allclose(Xg[live], fo[live], rtol=2e-3, atol=2e-3)
    np.testing.assert_allclose(Yg[live], yo[live], rtol=2e-3, atol=2e-3)
    np.testing.assert_allclose(ag, so * gas.rho0 * gas.c0 ** 2, rtol=2e-3, atol=1e-3 * ag.max())


def test_spherical_closure_absorbs_a_centred_pulse(cuda_device):
    """The memory on its own, through a network that realises w_in = psi:
    on the truncated ball a centred pulse leaves with far less reflected
    energy than under the characteristic condition (the large ball is the reference)."""
    nested = L.nested_ball(16)
    rc, _ = L.reflected_energy(3, nested, 0.01, 0.3, (0.0, 0.0, 0.0), B.DG_BC_CHARACTERISTIC)
    rs, _ = L.reflected_energy(3, nested, 0.01, 0.3, (0.0, 0.0, 0.0), B.DG_BC_LEARNED,
                               weights=L.spherical_weights())
    print("reflected energy, characteristic / spherical:", rc, rs)
    assert rs < 0.2 * rc


def test_learned_closure_against_characteristic_and_spherical(cuda_device):
    """Train on the method's own traces at r = 1 inside the radius-2 ball (the
    bench's seeded runs: 8 with random centres, 48 centred, an eighth of the
    trace nodes sampled, 1200 Adam iterations; the network without the
    absolute-direction inputs)
    and compare reflected energies on the truncated ball (the large ball is
    the reference) with the two conditions the network starts from or
    improves on:

    * the characteristic condition: the trained closure reflects far less,
      on centred and off-centre pulses;
    * the spherical-wave memory (the network's starting point, output zero):
      off the centre, where the memory's curvature is wrong, training
      reduces the reflection below the memory's (0.9x at most). On a
      centred pulse the memory is exact up to discretisation (~1e-5 of the
      energy); the network, which sees one face node's trace and cannot
      tell a centred wavefront from an off-centre one at the same
      incidence, adds a little of its fitting error there: it stays within
      1.3 times the memory's reflection (measured 0.8-1.05), three orders
      below the characteristic condition. The trained network has zero
      weights on the normal and position inputs."""
    p, n = 3, 16
    nested = L.nested_ball(n)
    X, Y = L.record(p, nested, L.run_seeds(0, 8, 48), every=10, device=cuda_device,
                    width_scale=2.0, node_fraction=0.125)
    assert X.shape[0] > 100000
    w, hist = L.train(X, Y, iters=1200, lr=3e-3, seed=0, radius=1.0, order=p)
    assert hist[-1] < 0.9 * hist[0]
    W1 = np.asarray(w)[:12 * 64].reshape(12, 64)
    assert np.all(W1[list(L.DIRECTION_FEATURES)] == 0.0)
    table = {}
    for amp, width, centre in ((0.005, 0.3, (0.0, 0.0, 0.0)), (0.1, 0.3, (0.0, 0.0, 0.0)),
                               (0.02, 0.25, (0.3, 0.1, -0.2)), (0.02, 0.25, (-0.2, 0.35, 0.1))):
        table[(amp, centre)] = L.reflection_table(p, nested, amp, width, centre, w)
    print("reflected energies:", table, "loss", hist[0], hist[-1])
    for (amp, centre), r in table.items():
        assert r["learned"] < 0.15 * r["characteristic"], (amp, centre, r)
        if centre == (0.0, 0.0, 0.0):
            assert r["learned"] < 1e-3 * r["characteristic"], (amp, centre, r)
            assert r["learned"] < 1.3 * r["spherical"], (amp, centre, r)
        else:
            assert r["learned"] < 0.9 * r["spherical"], (amp, centre, r)
