"""Degenerate and ragged sizes (GPU): a single tetrahedron (every face on
the boundary, one tile holding one element), two tetrahedra sharing a face
(in a shuffled vertex order), and meshes one element longer than a whole
number of tiles of each form (a last tile holding one element), against
the oracles at the bars of the other parity tests: float64 nodal and the
paper's modal form to 1e-11 per variable, float32 to 2e-5 of the
right-hand side and 2e-4 of the perturbation over a run."""
import numpy as np
import pytest

from oracle import modal_dg as MD
from paper_1710_03887_gb300 import workloads as W

from ._cases import SI, Case, rel_err, state_err

pytestmark = pytest.mark.gpu

FORMS = ["fp64", "f32", "f32_tc", "modal"]
TILE = {"fp64": 24, "f32": 32, "f32_tc": 25, "modal": 8}     # elements per tile at p = 2


def _meshes():
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 1.0, 1.0]])
    yield "one element", xyz, np.array([[0, 1, 2, 3]], dtype=np.int32)
    yield "two elements", xyz, np.array([[0, 1, 2, 3], [2, 3, 1, 4]], dtype=np.int32)


def _library(case, prec):
    from paper_1710_03887_gb300 import binding as B
    code = {"fp64": B.DG_PREC_FP64, "f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC,
            "modal": B.DG_PREC_MODAL}[prec]
    S = B.Solver(case.p, precision=code, **case.gas_kw)
    S.upload_mesh(case.xyz, case.EToV)
    return S


def _check(case, prec, steps=5):
    q = case.smooth(0.05, seed=1)
    if prec == "modal":
        orc = MD.ModalSolver(case.geom, case.gas)
        ref = orc.rhs_nodal(q)
    else:
        ref = case.oracle.rhs(q)
    S = _library(case, prec)
    S.set_state(q)
    err = rel_err(S.eval_rhs(), ref)
    assert np.all(err < (2e-5 if prec.startswith("f32") else 1e-11)), err
    q0 = case.pulse(0.02, 0.5, center=(0.2, 0.2, 0.2))
    dt = case.oracle.stable_dt(q0, 0.4)
    if prec == "modal":
        qo, _, _ = orc.run(q0, dt, steps)
    else:
        qo, _, _, _ = case.oracle.run(q0, dt, steps)
    S.set_state(q0)
    S.step(steps, dt)
    qg, _ = S.get_state()
    if prec.startswith("f32"):
        e = np.abs(qg - qo).max(axis=(0, 2)) / np.abs(qo - q0).max(axis=(0, 2))
        assert np.all(e < 2e-4), e
    else:
        assert np.all(state_err(qg, qo, case.gas) < 1e-11)


@pytest.mark.parametrize("prec", FORMS)
def test_one_and_two_elements(cuda_device, prec):
    for name, xyz, EToV in _meshes():
        _check(Case(2, xyz, EToV), prec)


@pytest.mark.parametrize("prec", FORMS)
def test_last_tile_holds_one_element(cuda_device, prec):
    xyz, EToV = W.kuhn_cube(2, jitter=0.1, seed=4)             # 48 elements
    keep = np.zeros(len(EToV), dtype=bool)
    keep[:TILE[prec] + 1] = True
    sx, sE = W.submesh(xyz, EToV, keep)
    _check(Case(2, sx, sE), prec)
