"""The largest workloads of the configurations, in the launch configuration
the bench uses: the 1,500,282-element p=3 cube lattice (float32 forms, the
mixed-precision configuration's size) and the 7,986,000-element p=4 cube
lattice (float32, the production configuration's size). Sampled elements'
right-hand sides are compared with the oracle evaluated on the patch made of
those elements and their neighbours.

Tolerance: on fine meshes the float32 rounding of the contractions is
relative to the terms before they cancel, sum |D| |F~'|, which grows like 1/h
against the derivative itself, so a fixed fraction of max |rhs| is not a
mesh-independent bound. Each node and variable is held to the dot-product
bound of its two float32 contractions plus the input rounding of the face
jumps, and the float64 oracle's own rounding (tests/_cases.f32_parity_bound)."""
import numpy as np
import pytest

from oracle import mlp as OM
from oracle.euler_dg import LEARNED, Gas
from oracle.euler_dg import Solver as OSolver
from oracle.geometry import Geometry
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import workloads as W

from ._cases import SI, f32_parity_bound

pytestmark = pytest.mark.gpu


def _device_pulse(S, xyz, EToV, order, dev, amplitude=0.05, width=0.3, chunk=1 << 20):
    """Pulse state on the device, built chunk by chunk on the host from the
    affine node map (node positions = barycentric weights of the reference
    nodes times the element's vertices)."""
    import torch
    ops = B.reference_operators(order)
    r, s, t = ops["r"], ops["s"], ops["t"]
    w = np.stack([-0.5 * (1 + r + s + t), 0.5 * (1 + r), 0.5 * (1 + s), 0.5 * (1 + t)])
    K = EToV.shape[0]
    q = torch.empty((K, 5, S.Np), dtype=torch.float64, device=dev)
    for k0 in range(0, K, chunk):
        k1 = min(K, k0 + chunk)
        nodes = np.einsum("kvd,vn->knd", xyz[EToV[k0:k1]], w)
        qc = W.gaussian_pulse_state(nodes, SI["gamma"], SI["rho0"], SI["p0"], amplitude, width,
                                    center=(0.1, -0.2, 0.15))
        q[k0:k1] = torch.from_numpy(qc).to(dev)
    return q, w


def _sampled_parity(S, xyz, EToV, order, q_dev, w, seed, mlp=None, mlp_delta=0.0):
    """Worst error / bound per node and variable at sampled elements. With
    ``mlp`` = (parameters, radius) every outer face takes the learned
    closure, and the bound adds what a network output off by ``mlp_delta``
    does to the oracle's right-hand side (the float32 network's error)."""
    rhs = S.eval_rhs()
    g = S.geometry()
    rng = np.random.default_rng(seed)
    K = EToV.shape[0]
    bdry = np.nonzero((g["EToE"] < 0).any(axis=1))[0]
    sample = np.unique(np.concatenate([rng.choice(K, 24, replace=False),
                                       rng.choice(bdry, 8, replace=False), [0, K - 1]]))
    patch = np.unique(np.concatenate([sample, g["EToE"][sample].ravel()]))
    patch = patch[patch >= 0]
    sub_xyz, sub_EToV = W.submesh(xyz, EToV, np.isin(np.arange(K), patch))
    geom = Geometry(ReferenceElement(order), sub_xyz, sub_EToV)
    gas = Gas(SI["gamma"], SI["rho0"], SI["p0"])
    kw = {} if mlp is None else dict(bc_mode={0: LEARNED}, mlp=mlp)
    osol = OSolver(geom, gas, **kw)
    import torch
    ro = osol.rhs(q_dev[torch.as_tensor(patch, device=q_dev.device)].cpu().numpy())
    local = np.searchsorted(patch, sample)
    assert np.array_equal(geom.boundary[local], g["EToE"][sample] < 0)
    qp = q_dev[torch.as_tensor(patch, device=q_dev.device)].cpu().numpy()
    bound = f32_parity_bound(osol, qp, gas)[local]
    if mlp is not None:
        # the network's output error: output 0 shifted by +-delta (b3[0])
        for sgn in (1.0, -1.0):
            wd = np.array(mlp[0], dtype=np.float64)
            wd[-5] += sgn * mlp_delta
            od = OSolver(geom, gas, bc_mode={0: LEARNED}, mlp=(wd, mlp[1]))
            bound = bound + 0.5 * np.abs(od.rhs(qp) - ro)[local]
    err = np.abs(rhs[sample] - ro[local])
    floor = 1e-7 * np.abs(ro[local]).max(axis=(0, 2))[None, :, None]
    ratio = err / (bound + floor)
    print("worst error / float32 bound per variable:", ratio.max(axis=(0, 2)))
    if mlp is None:
        return ratio
    # the same comparison against the characteristic condition's rhs: what
    # the test could not tell apart from the closure
    rc = OSolver(geom, gas).rhs(qp)
    ratio_char = np.abs(rhs[sample] - rc[local]) / (bound + floor)
    print("against the characteristic condition:", ratio_char.max(axis=(0, 2)))
    return ratio, ratio_char


@pytest.mark.parametrize("prec", [B.DG_PREC_F32, B.DG_PREC_F32_TC])
def test_c3_size_cube_p3(cuda_device, prec):
    xyz, EToV = W.kuhn_cube(63, jitter=0.1, seed=3)
    assert EToV.shape[0] == 1_500_282
    S = B.Solver(3, precision=prec, **SI)
    S.upload_mesh(xyz, EToV)
    q, w = _device_pulse(S, xyz, EToV, 3, cuda_device)
    S.set_state(q)
    ratio = _sampled_parity(S, xyz, EToV, 3, q, w, seed=1)
    assert np.all(ratio <= 1.0), ratio.max(axis=(0, 2))
    # and the state survives a few full steps at this size
    dt = S.stable_dt(q.cpu().numpy(), 0.5)
    S.step(5, dt)
    qe, _ = S.get_state(q)
    assert bool(qe.isfinite().all())


def test_c5_size_cube_p4(cuda_device):
    xyz, EToV = W.kuhn_cube(110, jitter=0.1, seed=5)
    assert EToV.shape[0] == 7_986_000
    S = B.Solver(4, precision=B.DG_PREC_F32, **SI)
    S.upload_mesh(xyz, EToV)
    q, w = _device_pulse(S, xyz, EToV, 4, cuda_device)
    S.set_state(q)
    ratio = _sampled_parity(S, xyz, EToV, 4, q, w, seed=2)
    assert np.all(ratio <= 1.0), ratio.max(axis=(0, 2))


def test_c5_size_cube_p4_learned_closure(cuda_device):
    """The production configuration's order and size with the learned
    closure on every outer face (seeded network, the memory at zero as after
    dg_set_state). Bound: the float32 stage's, plus the effect of a network
    output off by 2e-5 from the float64 one: the tensor-core GEMMs split
    their operands into tf32 head and tail (2^-22 relative per product,
    64-term sums of |h| <= 1 times weights of O(1): ~1.5e-5 at worst) and
    the hidden units' tanh is accurate to ~1e-7."""
    xyz, EToV = W.kuhn_cube(110, jitter=0.1, seed=5)
    rng = np.random.default_rng(11)
    w = OM.init_params(seed=11) + 0.05 * rng.normal(size=OM.N_PARAMS)
    w[-5 - 64 * 5:] *= 0.2
    S = B.Solver(4, precision=B.DG_PREC_F32, **SI)
    S.upload_mesh(xyz, EToV)
    S.set_bc(0, B.DG_BC_LEARNED)
    S.set_bc_mlp(w.astype(np.float32), 1.0)
    q, wn = _device_pulse(S, xyz, EToV, 4, cuda_device, width=0.8)     # reaches the faces
    S.set_state(q)
    ratio, ratio_char = _sampled_parity(S, xyz, EToV, 4, q, wn, seed=4,
                                        mlp=(w.astype(np.float32).astype(np.float64), 1.0),
                                        mlp_delta=2e-5)
    assert np.all(ratio <= 1.0), ratio.max(axis=(0, 2))
    assert ratio_char.max() > 10.0, ratio_char.max(axis=(0, 2))
