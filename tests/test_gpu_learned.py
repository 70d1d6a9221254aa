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
from oracle.euler_dg import learned_target
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


def test_learned_closure_rhs_matches_oracle(cuda_device):
    p = 2
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=4)
    gas = Gas(SI["gamma"], SI["rho0"], SI["p0"])
    ref = ReferenceElement(p)
    geom = Geometry(ref, xyz, EToV)
    w = _weights(5, out_scale=0.2)
    orc = OSolver(geom, gas, bc_mode={0: LEARNED}, mlp=(w, 1.3))
    q = W.random_smooth_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, seed=6)
    ro = orc.rhs(q)
    S = B.Solver(p, precision=B.DG_PREC_F32, **SI)
    S.upload_mesh(xyz, EToV)
    S.set_bc(0, B.DG_BC_LEARNED)
    S.set_bc_mlp(w.astype(np.float32), 1.3)
    S.set_state(q)
    err = rel_err(S.eval_rhs(), ro)
    assert np.all(err < 2e-5), err
    # the correction matters: the characteristic condition gives a different rhs
    orc_c = OSolver(geom, gas)
    assert np.abs(orc_c.rhs(q) - ro).max() > 1e-3 * np.abs(ro).max()


def test_trace_samples_match_oracle(cuda_device):
    import torch
    p = 2
    nested = L.nested_ball(8)
    S = B.Solver(p, precision=B.DG_PREC_F32, **SI)
    S.upload_mesh(*nested.big)
    elem, face = L.trace_faces(S, nested)
    assert len(elem) == 12 * 4 ** 2                 # the r = 1 sphere: 2 triangles per lattice square
    S.set_trace_faces(elem, face)
    ref = ReferenceElement(p)
    geom = Geometry(ref, *nested.big)
    gas = Gas(SI["gamma"], SI["rho0"], SI["p0"])
    q = W.random_smooth_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, seed=7)
    S.set_state(q)
    n = len(elem) * S.Nfp
    X = torch.empty((n, 12), dtype=torch.float32, device=cuda_device)
    Y = torch.empty((n, 5), dtype=torch.float32, device=cuda_device)
    S.sample_traces(X, Y)
    S.sync()
    # the same samples in float64 from the oracle's own pairing
    flat = np.transpose(q, (0, 2, 1)).reshape(-1, 5)
    qm = flat[geom.vmapM[elem, face]]                # [nf, Nfp, 5]
    qo = flat[geom.vmapP[elem, face]]
    nv = np.broadcast_to(geom.nrm[elem, face][:, None, :], qm.shape[:2] + (3,))
    xf = geom.x[elem[:, None], ref.Fmask[face]]
    q0 = gas.freestream()
    fo, s = OM.features(qm - q0, nv, xf, gas, 1.0)
    yo = learned_target(qm, qo, nv, gas)
    # features and targets are divided by the outgoing amplitude s, itself a
    # float32 sum p' + rho0 c0 u_n that partly cancels: relative tolerance
    np.testing.assert_allclose(X.cpu().numpy(), fo.reshape(-1, 12), rtol=1e-3, atol=2e-5)
    np.testing.assert_allclose(Y.cpu().numpy(), yo.reshape(-1, 5), rtol=1e-3, atol=2e-4)


def test_learned_closure_beats_characteristic(cuda_device):
    """Train on the method's own traces at r = 1 inside the radius-2 ball and
    compare reflected energies on the truncated ball (the large ball judges)."""
    p, n = 3, 16
    nested = L.nested_ball(n)
    runs = L.run_seeds(0, 6)
    X, Y = L.record(p, nested, runs, every=10, device=cuda_device, width_scale=2.0)
    assert X.shape[0] > 100000
    w, hist = L.train(X, Y, iters=600, lr=3e-3, seed=0, radius=1.0, order=p)
    assert hist[-1] < 0.5 * hist[0]
    gains = []
    for amp, width, centre in ((0.005, 0.3, (0.0, 0.0, 0.0)), (0.05, 0.3, (0.0, 0.0, 0.0)),
                               (0.02, 0.25, (0.3, 0.1, -0.2))):
        rc, _ = L.reflected_energy(p, nested, amp, width, centre, B.DG_BC_CHARACTERISTIC)
        rl, _ = L.reflected_energy(p, nested, amp, width, centre, B.DG_BC_LEARNED, weights=w)
        gains.append(rc / rl)
    print("reflected energy, characteristic / learned:", gains, "loss", hist[0], hist[-1])
    assert all(g > 1.05 for g in gains), gains
