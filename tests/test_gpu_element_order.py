"""Element order (GPU): the stage kernels tile runs of consecutive elements,
evaluate faces inside a tile once and gather across tiles, so the nodal
forms must give the same answer for any element order. A randomly permuted
mesh (no locality: almost no face inside a tile) and a Morton-sorted one
are run against the oracle and against the lattice-ordered run, permuted
back. The paper's discretisation integrates each interior face with the
Gauss rule of its lower-numbered element, so renumbering changes the rule
on some faces: each order is held to the modal oracle on the same
numbering, and the orders to each other at quadrature-error level."""
import numpy as np
import pytest

from paper_1710_03887_gb300 import workloads as W

from ._cases import SI, Case, rel_err, state_err

pytestmark = pytest.mark.gpu


def _solver(prec_name, p):
    from paper_1710_03887_gb300 import binding as B
    prec = {"fp64": B.DG_PREC_FP64, "f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC,
            "modal": B.DG_PREC_MODAL}[prec_name]
    return B.Solver(p, precision=prec, **SI)


@pytest.mark.parametrize("prec", ["fp64", "f32", "f32_tc", "modal"])
def test_any_element_order_gives_the_same_run(cuda_device, prec):
    p = 3
    xyz, EToV = W.kuhn_cube(5, jitter=0.1, seed=21)          # 750 elements, 24+ tiles
    base = Case(p, xyz, EToV)
    q0 = base.pulse(0.05, 0.3)
    dt = base.oracle.stable_dt(q0, 0.4)
    runs = {}
    for name, perm in (("lattice", np.arange(len(EToV))), ("morton", W.morton_order(xyz, EToV)),
                       ("random", W.random_order(len(EToV), 3))):
        S = _solver(prec, p)
        S.upload_mesh(xyz, EToV[perm])
        S.set_state(q0[perm])
        if name == "random" and prec == "fp64":
            # the permuted right-hand side against the oracle on the permuted
            # mesh, for a state whose every field has an O(1) right-hand side
            qs = base.smooth(0.05, seed=5)[perm]
            S.set_state(qs)
            ref = Case(p, xyz, EToV[perm]).oracle.rhs(qs)
            assert np.all(rel_err(S.eval_rhs(), ref) < 1e-11)
            S.set_state(q0[perm])
        S.step(10, dt)
        q, _ = S.get_state()
        if prec == "modal":
            from oracle.modal_dg import ModalSolver
            qo, _, _ = ModalSolver(Case(p, xyz, EToV[perm]).geom, base.gas).run(q0[perm], dt, 10)
            assert np.all(state_err(q, qo, base.gas) < 1e-11), name
        out = np.empty_like(q)
        out[perm] = q
        runs[name] = out
    base_q = runs["lattice"]
    for name in ("morton", "random"):
        if prec == "fp64":
            err = state_err(runs[name], base_q, base.gas)
            assert np.all(err < 1e-12), (name, err)
        elif prec == "modal":
            pert = np.abs(base_q - q0).max(axis=(0, 2))
            err = np.abs(runs[name] - base_q).max(axis=(0, 2)) / pert
            assert np.all(err < 1e-3), (name, err)        # another Gauss rule on some faces
        else:
            # float32: the tile split changes the order of roundings only
            pert = np.abs(base_q - q0).max(axis=(0, 2))
            err = np.abs(runs[name] - base_q).max(axis=(0, 2)) / pert
            assert np.all(err < 1e-4), (name, err)
