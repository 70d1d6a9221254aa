"""The horn-in-room workload on the GPU (GPU): a flared horn with slip walls,
driven by the inflow pulse of section 2.4 at its mouthpiece, inside a
pass-through room (the domain types of section 1.2: a room in front of the
bell only, at the mixed-precision configuration's size of ~1.5 M elements,
or a room enclosing the whole horn).

* small horns (4,464 elements in front of the bell, 12,432 enclosing; p = 2):
  every form against the oracle over 16 steps in which one whole inflow
  pulse enters: float64 to 1e-11 per variable, float32 forms to 2e-4 of the
  perturbation (the tolerances of the other run tests, same reasoning);
* full size (1,489,704 elements, p = 3, float32): sampled right-hand sides
  against the oracle on the patch around them (walls, rim, mouthpiece and
  room elements included), each node held to the float32 form's rounding
  bound plus the oracle's own (at rest the float32 form computes exact
  zeros where the float64 oracle leaves rounding of the base state);
  then a run with the inflow pulse, mass balanced against the boundary-flux
  ledger, and the sensor analogues of Table 2 located and read."""
import functools

import numpy as np
import pytest

from oracle.euler_dg import CHARACTERISTIC, INFLOW_PULSE, SLIP_WALL, Gas
from oracle.euler_dg import Solver as OSolver
from oracle.geometry import Geometry
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import workloads as W

from ._cases import SI, f32_parity_bound

pytestmark = pytest.mark.gpu

SMALL = dict(m1=1, room_length=0.03, room_half=0.03, growth=1.8, horn_length=0.1, aspect=3.0)
DOMAINS = {"bell-front": SMALL, "enclosing": dict(SMALL, behind=0.02)}
MODES = {W.HORN_OUTER: CHARACTERISTIC, W.HORN_WALL: SLIP_WALL, W.HORN_MOUTHPIECE: INFLOW_PULSE}
LIB_MODES = {W.HORN_OUTER: B.DG_BC_CHARACTERISTIC, W.HORN_WALL: B.DG_BC_SLIP_WALL,
             W.HORN_MOUTHPIECE: B.DG_BC_INFLOW_PULSE}
PRECS = {"fp64": B.DG_PREC_FP64, "f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC}
GAS = Gas(SI["gamma"], SI["rho0"], SI["p0"])


def _oracle(p, xyz, EToV, tag):
    geom = Geometry(ReferenceElement(p), xyz, EToV)
    return OSolver(geom, GAS, bc_id=np.where(tag < 0, 0, tag).astype(np.int64), bc_mode=MODES)


def _library(p, prec, xyz, EToV, tag, amp, alpha):
    S = B.Solver(p, precision=PRECS[prec], **SI)
    S.upload_mesh(xyz, EToV, face_tag=tag)
    for ident, mode in LIB_MODES.items():
        S.set_bc(ident, mode)
    S.set_inflow(amp, alpha)
    return S


@functools.lru_cache(maxsize=None)
def _oracle_run(domain):
    """16 oracle steps from rest with one whole inflow pulse (shared by the forms)."""
    xyz, EToV, tag, _ = W.horn_in_room(**DOMAINS[domain])
    orc = _oracle(2, xyz, EToV, tag)
    q0 = W.uniform_state(orc.g.K, orc.ref.Np, SI["rho0"], (0, 0, 0), SI["p0"], SI["gamma"])
    dt = orc.stable_dt(q0, 0.5)
    alpha = 2 * np.pi / (12 * dt)
    orc.inflow = (0.1, alpha)
    qo, _, ledger_o, _ = orc.run(q0, dt, 16)
    return xyz, EToV, tag, q0, dt, alpha, qo, ledger_o


@pytest.mark.parametrize("domain", list(DOMAINS))
@pytest.mark.parametrize("prec", list(PRECS))
def test_small_horn_inflow_run_matches_oracle(cuda_device, prec, domain):
    xyz, EToV, tag, q0, dt, alpha, qo, ledger_o = _oracle_run(domain)
    p = 2
    S = _library(p, prec, xyz, EToV, tag, 0.1, alpha)
    S.set_state(q0)
    tot0 = S.totals()
    S.step(16, dt)
    qg, _ = S.get_state()
    pert = np.abs(qo - q0).max(axis=(0, 2))
    assert np.all(pert[[0, 1, 4]] > 0)                  # the pulse entered
    if prec == "fp64":
        err = np.abs(qg - qo).max(axis=(0, 2)) / np.abs(qo).max(axis=(0, 2))
        assert np.all(err < 1e-11), err
    else:
        pert[1:4] = pert[1:4].max()                     # momentum: relative to its largest component
        err = np.abs(qg - qo).max(axis=(0, 2)) / pert
        assert np.all(err < 2e-4), err
    # mass entered through the mouthpiece only (walls carry no mass flux)
    led = S.boundary_flux()
    bal = S.totals() - tot0 + led
    assert abs(bal[0]) <= 1e-9 * abs(tot0[0]) + 1e-3 * abs(ledger_o[0])
    assert led[0] == pytest.approx(ledger_o[0], rel=1e-9 if prec == "fp64" else 1e-3)


def _device_pulse(S, xyz, EToV, order, dev, center, width, amplitude, chunk=1 << 20):
    import torch
    ops = B.reference_operators(order)
    r, s, t = ops["r"], ops["s"], ops["t"]
    w = np.stack([-0.5 * (1 + r + s + t), 0.5 * (1 + r), 0.5 * (1 + s), 0.5 * (1 + t)])
    K = EToV.shape[0]
    q = torch.empty((K, 5, S.Np), dtype=torch.float64, device=dev)
    for k0 in range(0, K, chunk):
        k1 = min(K, k0 + chunk)
        nodes = np.einsum("kvd,vn->knd", xyz[EToV[k0:k1]], w)
        q[k0:k1] = torch.from_numpy(W.gaussian_pulse_state(
            nodes, SI["gamma"], SI["rho0"], SI["p0"], amplitude, width, center=center)).to(dev)
    return q


def test_full_size_horn_sampled_parity_run_and_sensors(cuda_device):
    import torch
    xyz, EToV, tag, info = W.horn_in_room()
    K = EToV.shape[0]
    assert K == 1_489_704
    S = _library(3, "f32", xyz, EToV, tag, 0.1, 2 * np.pi * 2000.0)
    # a pulse straddling the bell plane: horn, rim and room elements all see it
    q = _device_pulse(S, xyz, EToV, 3, cuda_device, (info["bell_x"], 0.02, 0.0), 0.03, 0.05)
    S.set_state(q)
    rhs = S.eval_rhs()
    rng = np.random.default_rng(7)
    kinds = [np.nonzero(np.any(tag == b, axis=1))[0] for b in (W.HORN_WALL, W.HORN_MOUTHPIECE, W.HORN_OUTER)]
    cent = xyz[EToV].mean(axis=1)
    near = np.nonzero(np.linalg.norm(cent - [info["bell_x"], 0.02, 0.0], axis=1) < 0.03)[0]
    sample = np.unique(np.concatenate([rng.choice(K, 16, replace=False), rng.choice(near, 24, replace=False)]
                                      + [rng.choice(k, 8, replace=False) for k in kinds]))
    g = S.geometry()
    patch = np.unique(np.concatenate([sample, g["EToE"][sample].ravel()]))
    patch = patch[patch >= 0]
    sub_xyz, sub_EToV = W.submesh(xyz, EToV, np.isin(np.arange(K), patch))
    orc = _oracle(3, sub_xyz, sub_EToV, tag[patch])
    local = np.searchsorted(patch, sample)
    assert np.array_equal(orc.g.boundary[local], tag[sample] >= 0)
    qp = q[torch.as_tensor(patch, device=q.device)].cpu().numpy()
    ro = orc.rhs(qp, 0.0)
    bound = f32_parity_bound(orc, qp, GAS)[local]
    err = np.abs(rhs[sample] - ro[local])
    floor = 1e-7 * np.abs(ro[local]).max(axis=(0, 2))[None, :, None]
    ratio = err / (bound + floor)
    worst = np.argsort(-ratio.max(axis=(1, 2)))[:6]
    for i in worst:
        e = sample[i]
        print("element", e, "tags", tag[e], "centroid", np.round(cent[e], 4),
              "ratio", ratio[i].max(axis=1), "lib", np.abs(rhs[e]).max(axis=1),
              "oracle", np.abs(ro[local[i]]).max(axis=1), "bound", bound[i].max(axis=1))
    assert np.all(ratio <= 1.0), ratio.max(axis=(0, 2))
    # run: the inflow pulse enters, the bell pulse spreads; mass balances the ledger
    S.set_probes(info["sensors"], capacity=64)
    S.set_state(q)
    tot0 = S.totals()
    dt = S.stable_dt(q.cpu().numpy(), 0.5)
    S.step(40, dt)
    qe, t = S.get_state(q)
    assert bool(qe.isfinite().all()) and t == pytest.approx(40 * dt)
    bal = S.totals() - tot0 + S.boundary_flux()
    assert abs(bal[0]) <= 1e-6 * abs(tot0[0]), bal
    series = S.read_probes(40)
    assert series.shape == (40, 4, 5)
    # the sensors are far from both pulses: the air there is still at rest
    assert np.allclose(series[:, :, 0], SI["rho0"], rtol=1e-6)
