"""The paper's own discretisation on the GPU (DG_PREC_MODAL) against its
oracle (oracle/modal_dg.py), element by element (GPU).

Both compute the same polynomials in float64 (the library on nodal values
with the orthonormal basis folded into its operators, the oracle on modal
coefficients), so the bound is the float64 path's: per conserved variable,
max |gpu - oracle| / scale <= 1e-11, the scale as in the nodal parity tests
(max |oracle| for density and energy, rho0 c0 for momentum)."""
import numpy as np
import pytest

from oracle import modal_dg as MD
from oracle.euler_dg import Gas
from oracle.geometry import Geometry
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import workloads as W

from ._cases import (CHARACTERISTIC, FREESTREAM, SI, SLIP_WALL, direction_tags, rel_err,
                     state_err)

pytestmark = pytest.mark.gpu

TOL = 1e-11
GAS = Gas(SI["gamma"], SI["rho0"], SI["p0"])


def _library(p, xyz, EToV, tags=None, modes=None, vclass=None):
    from paper_1710_03887_gb300 import binding as B
    S = B.Solver(p, precision=B.DG_PREC_MODAL, **SI)
    S.upload_mesh(xyz, EToV, face_tag=tags, vert_class=vclass)
    for ident, mode in (modes or {}).items():
        S.set_bc(ident, mode)
    return S


def _mixed(p, seed):
    xyz, EToV = W.kuhn_cube(3, jitter=0.12, seed=seed)
    geom = Geometry(ReferenceElement(p), xyz, EToV)
    tags = direction_tags(xyz, EToV, geom)
    modes = {0: CHARACTERISTIC, 1: FREESTREAM, 2: SLIP_WALL}
    orc = MD.ModalSolver(geom, GAS, bc_id=np.where(tags < 0, 0, tags), bc_mode=modes)
    return xyz, EToV, geom, tags, modes, orc


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_modal_rhs_matches_oracle_mixed_boundaries(cuda_device, p):
    xyz, EToV, geom, tags, modes, orc = _mixed(p, p)
    q = W.random_smooth_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, seed=p)
    ref = orc.rhs_nodal(q)
    S = _library(p, xyz, EToV, tags, modes)
    S.set_state(q)
    err = rel_err(S.eval_rhs(), ref)
    assert np.all(err < TOL), err


@pytest.mark.parametrize("p", [1, 2])
def test_modal_pulse_run_and_ledger(cuda_device, p):
    """The paper's configuration (p = 1, RK2; p = 2 as its check): a pulse
    on the 1296-element cube with the characteristic condition, 40 Heun
    steps; state and boundary-flux ledger against the oracle."""
    xyz, EToV = W.kuhn_cube(6)
    geom = Geometry(ReferenceElement(p), xyz, EToV)
    orc = MD.ModalSolver(geom, GAS)
    q0 = W.gaussian_pulse_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.005, 0.15)
    from oracle.euler_dg import Solver
    dt = Solver(geom, GAS).stable_dt(q0, 0.3)
    qo, _, led_o = orc.run(q0, dt, 40)
    S = _library(p, xyz, EToV)
    S.set_state(q0)
    tot0 = S.totals()
    S.step(40, dt)
    qg, t = S.get_state()
    assert t == pytest.approx(40 * dt)
    err = state_err(qg, qo, GAS)
    assert np.all(err < TOL), err
    # ledger against the oracle's, relative to the flux scale (as the nodal tests)
    led = S.boundary_flux()
    assert np.allclose(led, led_o, rtol=1e-9, atol=1e-12 * np.abs(tot0).max())
    bal = S.totals() - tot0 + led
    assert np.all(np.abs(bal) <= 1e-12 * np.maximum(np.abs(tot0), 1.0)), bal


def test_modal_inflow_horn_run(cuda_device):
    """Inflow pulse, slip walls and the characteristic room on the small
    horn (4,464 elements, p = 2), 12 Heun steps with one whole pulse."""
    from oracle.euler_dg import CHARACTERISTIC as CH, INFLOW_PULSE, SLIP_WALL as SW, Solver
    from paper_1710_03887_gb300 import binding as B
    xyz, EToV, tag, _ = W.horn_in_room(m1=1, room_length=0.03, room_half=0.03, growth=1.8,
                                       horn_length=0.1, aspect=3.0)
    geom = Geometry(ReferenceElement(2), xyz, EToV)
    q0 = W.uniform_state(geom.K, geom.ref.Np, SI["rho0"], (0, 0, 0), SI["p0"], SI["gamma"])
    dt = Solver(geom, GAS).stable_dt(q0, 0.3)
    alpha = 2 * np.pi / (10 * dt)
    modes = {W.HORN_OUTER: CH, W.HORN_WALL: SW, W.HORN_MOUTHPIECE: INFLOW_PULSE}
    orc = MD.ModalSolver(geom, GAS, bc_id=np.where(tag < 0, 0, tag), bc_mode=modes,
                         inflow=(0.1, alpha))
    qo, _, led_o = orc.run(q0, dt, 12)
    S = _library(2, xyz, EToV, tag, {W.HORN_OUTER: B.DG_BC_CHARACTERISTIC,
                                     W.HORN_WALL: B.DG_BC_SLIP_WALL,
                                     W.HORN_MOUTHPIECE: B.DG_BC_INFLOW_PULSE})
    S.set_inflow(0.1, alpha)
    S.set_state(q0)
    tot0 = S.totals()
    S.step(12, dt)
    qg, _ = S.get_state()
    assert np.abs(qo - q0).max() > 0
    err = state_err(qg, qo, GAS)
    assert np.all(err < TOL), err
    led = S.boundary_flux()
    assert np.allclose(led, led_o, rtol=1e-9, atol=1e-12 * np.abs(tot0).max())


def test_modal_periodic_conservation(cuda_device):
    """Fully periodic cube (no outer face): every total stays constant to
    rounding over 30 Heun steps, and the state follows the oracle."""
    p = 2
    xyz, EToV = W.kuhn_cube(4, jitter=0.1, seed=7)
    geom = Geometry(ReferenceElement(p), xyz, EToV, period=(2.0, 2.0, 2.0))
    q0 = W.random_smooth_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, seed=4)
    from oracle.euler_dg import Solver
    dt = Solver(geom, GAS).stable_dt(q0, 0.3)
    qo, _, _ = MD.ModalSolver(geom, GAS).run(q0, dt, 30)
    S = _library(p, xyz, EToV, vclass=W.periodic_vertex_classes(4))
    S.set_state(q0)
    tot0 = S.totals()
    S.step(30, dt)
    qg, _ = S.get_state()
    assert np.all(state_err(qg, qo, GAS) < TOL)
    np.testing.assert_allclose(S.totals(), tot0, rtol=0, atol=1e-13 * np.abs(tot0).max())
    assert np.all(S.boundary_flux() == 0.0)


def test_modal_full_size_p1_sampled_rhs(cuda_device):
    """The paper's configuration: p = 1 on the 196,608-element ball. Sampled
    elements' right-hand sides against the modal oracle on the patch made of
    them and their neighbours (the patch keeps the elements' relative order,
    so every face keeps the Gauss rule of its lower-numbered element)."""
    import torch
    xyz, EToV = W.ball(32, 1.0, jitter=0.1, seed=0)
    K = EToV.shape[0]
    S = _library(1, xyz, EToV)
    q = W.random_smooth_state(S.node_coords(), SI["gamma"], SI["rho0"], SI["p0"], 0.05, seed=9)
    S.set_state(q)
    rhs = S.eval_rhs()
    g = S.geometry()
    rng = np.random.default_rng(4)
    bdry = np.nonzero((g["EToE"] < 0).any(axis=1))[0]
    sample = np.unique(np.concatenate([rng.choice(K, 40, replace=False), rng.choice(bdry, 12, replace=False)]))
    patch = np.unique(np.concatenate([sample, g["EToE"][sample].ravel()]))
    patch = patch[patch >= 0]
    sx, sE = W.submesh(xyz, EToV, np.isin(np.arange(K), patch))
    orc = MD.ModalSolver(Geometry(ReferenceElement(1), sx, sE), GAS)
    local = np.searchsorted(patch, sample)
    ro = orc.rhs_nodal(q[patch])[local]
    # every field varies, so every variable's right-hand side is O(1)
    err = np.abs(rhs[sample] - ro).max(axis=(0, 2)) / np.abs(ro).max(axis=(0, 2))
    assert np.all(err < TOL), err


def test_modal_bad_state_is_reported_and_the_context_stays_usable(cuda_device):
    from paper_1710_03887_gb300 import binding as B
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=2)
    geom = Geometry(ReferenceElement(2), xyz, EToV)
    q0 = W.gaussian_pulse_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, 0.3)
    from oracle.euler_dg import Solver
    dt = Solver(geom, GAS).stable_dt(q0, 0.3)
    S = _library(2, xyz, EToV)
    S.set_state(q0)
    S.step(3, dt)
    ref, _ = S.get_state()
    bad = q0.copy()
    bad[7, 4, :] = 0.0                       # zero energy: negative pressure at every point
    S.set_state(bad)
    with pytest.raises(B.DGError) as e:
        S.step(1, dt)
        S.get_state()
    assert e.value.code == B.DG_ERR_NONFINITE
    S.set_state(q0)
    S.step(3, dt)
    q, _ = S.get_state()
    assert np.array_equal(q, ref)            # same bits as before the bad state
