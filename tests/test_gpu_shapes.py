"""The outer domains of section 1.2 (Table 1) on the GPU: small versions of
the hemisphere and the 45-degree cone in front of the bell (type B), and the
sphere, cone and spherical cone around the whole horn (type A), each with
the horn's slip walls, the inflow pulse at its mouthpiece and the
characteristic pass-through condition on the outer surface.

Every form against its oracle over 8 steps in which the inflow pulse enters
(p = 2): the nodal forms against the nodal oracle (float64 to 1e-11 per
variable, float32 forms to 2e-4 of the perturbation, the tolerances of the
other run tests), the paper's discretisation against the modal oracle
(1e-11). The boundary ledger agrees with the oracle's (mass enters through
the mouthpiece only) and the GPU's totals balance against it."""
import functools

import numpy as np
import pytest

from oracle import modal_dg as MD
from oracle.euler_dg import CHARACTERISTIC, INFLOW_PULSE, SLIP_WALL, Gas
from oracle.euler_dg import Solver as OSolver
from oracle.geometry import Geometry
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import workloads as W

from ._cases import SI, state_err

pytestmark = pytest.mark.gpu

SMALL = dict(m1=1, room_length=0.03, room_half=0.03, growth=1.8, horn_length=0.1, aspect=3.0)
ENCL = dict(SMALL, behind=0.03, growth=3.0, aspect=5.0)
SHAPES = {
    "B-half-sphere": dict(SMALL, shape="sphere"),
    "B-half-cone": dict(SMALL, shape="cone"),
    "A-sphere": dict(ENCL, shape="sphere"),
    "A-cone": dict(ENCL, shape="cone", room_half=0.06),
    "A-scone": dict(ENCL, shape="scone", room_half=0.06),
}
MODES = {W.HORN_OUTER: CHARACTERISTIC, W.HORN_WALL: SLIP_WALL, W.HORN_MOUTHPIECE: INFLOW_PULSE}
LIB_MODES = {W.HORN_OUTER: B.DG_BC_CHARACTERISTIC, W.HORN_WALL: B.DG_BC_SLIP_WALL,
             W.HORN_MOUTHPIECE: B.DG_BC_INFLOW_PULSE}
PRECS = {"fp64": B.DG_PREC_FP64, "f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC,
         "modal": B.DG_PREC_MODAL}
GAS = Gas(SI["gamma"], SI["rho0"], SI["p0"])
P, STEPS = 2, 8


@functools.lru_cache(maxsize=None)
def _mesh(name):
    xyz, EToV, tag, info = W.horn_in_room(**SHAPES[name])
    assert info["name"] == name
    geom = Geometry(ReferenceElement(P), xyz, EToV)
    q0 = W.uniform_state(geom.K, geom.ref.Np, SI["rho0"], (0, 0, 0), SI["p0"], SI["gamma"])
    bc_id = np.where(tag < 0, 0, tag).astype(np.int64)
    dt = OSolver(geom, GAS, bc_id=bc_id, bc_mode=MODES).stable_dt(q0, 0.3)
    alpha = 2 * np.pi / (10 * dt)                 # the pulse enters within the run
    return xyz, EToV, tag, geom, bc_id, q0, dt, alpha


@functools.lru_cache(maxsize=None)
def _oracle_run(name, modal):
    xyz, EToV, tag, geom, bc_id, q0, dt, alpha = _mesh(name)
    if modal:
        qo, _, led = MD.ModalSolver(geom, GAS, bc_id=bc_id, bc_mode=MODES,
                                    inflow=(0.1, alpha)).run(q0, dt, STEPS)
    else:
        orc = OSolver(geom, GAS, bc_id=bc_id, bc_mode=MODES)
        orc.inflow = (0.1, alpha)
        qo, _, led, _ = orc.run(q0, dt, STEPS)
    return qo, led


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("name", list(SHAPES))
def test_shape_inflow_run_matches_oracle(cuda_device, name, prec):
    xyz, EToV, tag, geom, _, q0, dt, alpha = _mesh(name)
    qo, led_o = _oracle_run(name, prec == "modal")
    S = B.Solver(P, precision=PRECS[prec], **SI)
    S.upload_mesh(xyz, EToV, face_tag=tag)
    for ident, mode in LIB_MODES.items():
        S.set_bc(ident, mode)
    S.set_inflow(0.1, alpha)
    S.set_state(q0)
    tot0 = S.totals()
    S.step(STEPS, dt)
    qg, _ = S.get_state()
    pert = np.abs(qo - q0).max(axis=(0, 2))
    assert np.all(pert[[0, 1, 4]] > 0)                  # the pulse entered
    if prec in ("fp64", "modal"):
        err = state_err(qg, qo, GAS)
        assert np.all(err < 1e-11), err
    else:
        pert[1:4] = pert[1:4].max()
        err = np.abs(qg - qo).max(axis=(0, 2)) / pert
        assert np.all(err < 2e-4), err
    led = S.boundary_flux()
    bal = S.totals() - tot0 + led
    assert abs(bal[0]) <= 1e-9 * abs(tot0[0]) + 1e-3 * abs(led_o[0])
    assert led[0] == pytest.approx(led_o[0], rel=1e-9 if prec in ("fp64", "modal") else 1e-3)
