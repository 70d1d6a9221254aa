"""Every vertex correspondence between the two sides of a face (GPU).

Lattice meshes list the vertices of a shared face in related orders, so
only some of the six orientation codes occur in them; mesh generators give
no such guarantee. Here each element's vertex list is shuffled (positively
oriented), so all six occur, and every form is held to its oracle at the
bars of the other parity tests: float64 nodal and the paper's modal form
to 1e-11 per variable, float32 (SIMT and tensor-core contractions) to the
float32 right-hand-side bound. The float32 forms evaluate a face inside a
tile once and write the neighbour's jump through the face-node table, so
this also covers that table in every orientation. The host-side pairing
itself is checked on the CPU against the oracle's coordinate matching
(tests/test_host_library.py)."""
import numpy as np
import pytest

from oracle import modal_dg as MD
from paper_1710_03887_gb300 import workloads as W

from ._cases import CHARACTERISTIC, FREESTREAM, SI, SLIP_WALL, Case, direction_tags, orientation_codes, rel_err, state_err

pytestmark = pytest.mark.gpu


def _shuffled_case(p, seed):
    xyz, EToV = W.kuhn_cube(3, jitter=0.12, seed=seed)
    E = W.shuffle_vertices(xyz, EToV, seed=seed + 100)
    probe = Case(p, xyz, E)
    g = probe.geom
    codes = orientation_codes(E, np.where(g.boundary, -1, g.EToE), g.EToF)[~g.boundary]
    assert set(codes.tolist()) == set(range(6))
    tags = direction_tags(xyz, E, g)
    return Case(p, xyz, E, tags=tags, modes={0: CHARACTERISTIC, 1: FREESTREAM, 2: SLIP_WALL})


def _library(case, prec):
    from paper_1710_03887_gb300 import binding as B
    code = {"fp64": B.DG_PREC_FP64, "f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC,
            "modal": B.DG_PREC_MODAL}[prec]
    S = B.Solver(case.p, precision=code, **case.gas_kw)
    S.upload_mesh(case.xyz, case.EToV, face_tag=case.tags)
    for ident, mode in case.modes.items():
        S.set_bc(ident, mode)
    return S


def _modal_oracle(case):
    return MD.ModalSolver(case.geom, case.gas, bc_id=np.where(case.tags < 0, 0, case.tags),
                          bc_mode=case.modes)


@pytest.mark.parametrize("prec,p", [("fp64", 2), ("fp64", 3), ("f32", 3), ("f32", 4),
                                    ("f32_tc", 3), ("f32_tc", 4), ("modal", 2), ("modal", 3)])
def test_rhs_in_every_orientation(cuda_device, prec, p):
    case = _shuffled_case(p, seed=30 + p)
    q = case.smooth(0.05, seed=p)
    ref = _modal_oracle(case).rhs_nodal(q) if prec == "modal" else case.oracle.rhs(q)
    S = _library(case, prec)
    S.set_state(q)
    err = rel_err(S.eval_rhs(), ref)
    assert np.all(err < (2e-5 if prec.startswith("f32") else 1e-11)), err


@pytest.mark.parametrize("prec", ["fp64", "f32", "modal"])
def test_pulse_run_in_every_orientation(cuda_device, prec):
    """Ten steps of an off-centre pulse (characteristic, free-stream and wall
    faces): float64 forms to 1e-11 of the state, float32 to 2e-4 of the
    perturbation (the bars of the other run tests)."""
    p = 3
    case = _shuffled_case(p, seed=40)
    q0 = case.pulse(0.05, 0.3, center=(0.2, -0.1, 0.1))
    dt = case.oracle.stable_dt(q0, 0.4)
    if prec == "modal":
        qo, _, _ = _modal_oracle(case).run(q0, dt, 10)
    else:
        qo, _, _, _ = case.oracle.run(q0, dt, 10)
    S = _library(case, prec)
    S.set_state(q0)
    S.step(10, dt)
    qg, _ = S.get_state()
    if prec == "f32":
        err = np.abs(qg - qo).max(axis=(0, 2)) / np.abs(qo - q0).max(axis=(0, 2))
        assert np.all(err < 2e-4), err
    else:
        assert np.all(state_err(qg, qo, case.gas) < 1e-11)
