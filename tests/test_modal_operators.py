"""The operators of the library's DG_PREC_MODAL form, built in C++ on the
host, checked without a GPU: a numpy transcription of the stage kernel's
algorithm (stage_modal.cu) with those operators, the oracle's geometry and
its coordinate-matched face nodes must reproduce the modal oracle's
right-hand side. This pins the operator algebra (orthonormal mass matrix
folded into nodal operators, Lagrange values at the Gauss points) and the
one-point-set-per-face convention (variant 0 below the neighbour's index,
1 + orientation code above it)."""
import numpy as np
import pytest

from oracle import modal_dg as MD
from oracle.euler_dg import (CHARACTERISTIC, FREESTREAM, GHOSTS, INFLOW_PULSE, SLIP_WALL, Gas,
                             euler_fluxes, ghost_inflow, llf_flux)
from oracle.geometry import Geometry
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import workloads as W

from ._cases import SI, direction_tags, orientation_codes

GAS = Gas(SI["gamma"], SI["rho0"], SI["p0"])


def _kernel_rhs(ops, geom, EToV, q, bc_id, modes, t=0.0, inflow=(0.05, 565.0)):
    g, ref = geom, geom.ref
    K, Np = g.K, ref.Np
    EToE = np.where(g.boundary, -1, g.EToE)
    ori = orientation_codes(EToV, EToE, g.EToF)
    var = np.where((EToE < 0) | (np.arange(K)[:, None] <= EToE), 0, 1 + ori)    # [K, 4]
    flat = np.transpose(q, (0, 2, 1)).reshape(K * Np, 5)
    um, up = flat[g.vmapM], flat[g.vmapP]                                     # [K, 4, Nfp, 5]
    Ifn = ops["Ifn"][np.arange(4)[None, :], var]                              # [K, 4, Nfq, Nfp]
    qm = np.einsum("kfqm,kfmv->kfqv", Ifn, um)
    qp = np.einsum("kfqm,kfmv->kfqv", Ifn, up)
    n = np.broadcast_to(g.nrm[:, :, None, :], qm.shape[:3] + (3,))
    for ident, mode in modes.items():
        sel = np.nonzero(g.boundary & (bc_id == ident))
        if mode == INFLOW_PULSE:
            qp[sel] = ghost_inflow(qm[sel], n[sel], GAS, t, *inflow)
        else:
            qp[sel] = GHOSTS[mode](qm[sel], n[sel], GAS)
    Fs = g.Fscale[:, :, None, None] * llf_flux(qm, qp, n, GAS.gamma)          # [K, 4, Nfq, 5]
    Uq = np.einsum("qn,kvn->kqv", ops["Iq"], q)
    F = np.stack(euler_fluxes(Uq, GAS.gamma), axis=1)                         # [K, 3 (x), Nq, 5]
    G = np.einsum("kad,kdqv->kaqv", g.drdx, F)                                # [K, 3 (r), Nq, 5]
    Sf = ops["Sf"][np.arange(4)[None, :], var]                                # [K, 4, Np, Nfq]
    rhs = np.einsum("anq,kaqv->kvn", ops["Sv"], G) - np.einsum("kfnq,kfqv->kvn", Sf, Fs)
    # float64 rounding bound of the two sums, from the size of their terms
    # before they cancel (the base pressure's volume and surface integrals
    # cancel to ~1/h of their size on small elements): (N + 10) u sum |terms|
    # and the rounding of the traces inside the LLF jump lambda (q+ - q-) / 2,
    # which is all that is left where the exact jump vanishes
    def speed(u):
        vel = u[..., 1:4] / u[..., :1]
        pr = (GAS.gamma - 1.0) * (u[..., 4] - 0.5 * u[..., 0] * np.sum(vel * vel, axis=-1))
        return np.abs(np.einsum("kfqd,kfqd->kfq", vel, n)) + np.sqrt(GAS.gamma * np.abs(pr) / u[..., 0])
    jump = 0.5 * np.maximum(speed(qm), speed(qp))[..., None] * (np.abs(qm) + np.abs(qp))
    mag = (np.einsum("anq,kaqv->kvn", np.abs(ops["Sv"]), np.abs(G))
           + np.einsum("kfnq,kfqv->kvn", np.abs(Sf), np.abs(Fs) + g.Fscale[:, :, None, None] * jump))
    N = 3 * ops["Iq"].shape[0] + 4 * ops["wf"].shape[0]
    return rhs, (N + 10) * 2.0 ** -53 * mag


@pytest.mark.parametrize("p,shuffled", [(1, False), (2, False), (3, False), (4, False),
                                        (2, True), (3, True)])
def test_library_operators_reproduce_the_modal_oracle(p, shuffled):
    """Lattice vertex lists, and shuffled ones where every orientation code
    (every variant 1 + o of the face operators) occurs."""
    xyz, EToV = W.kuhn_cube(3, jitter=0.12, seed=10 + p)
    if shuffled:
        EToV = W.shuffle_vertices(xyz, EToV, seed=20 + p)
    geom = Geometry(ReferenceElement(p), xyz, EToV)
    tags = direction_tags(xyz, EToV, geom)
    bc_id = np.where(tags < 0, 0, tags)
    modes = {0: CHARACTERISTIC, 1: FREESTREAM, 2: SLIP_WALL}
    q = W.random_smooth_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, seed=p)
    ref = MD.ModalSolver(geom, GAS, bc_id=bc_id, bc_mode=modes).rhs_nodal(q)
    got, bound = _kernel_rhs(B.modal_operators(p), geom, EToV, q, bc_id, modes)
    err = np.abs(got - ref).max(axis=(0, 2)) / np.abs(ref).max(axis=(0, 2))
    assert np.all(err < 1e-11), err                  # the float64 parity bar; measured <= 1.3e-12
    # both sides' rounding: the emulation's sums, and the oracle's own (its
    # conversions between nodal values and coefficients, condition <= 16,
    # add rounding of the same order); measured <= 2.5 bounds
    assert np.all(np.abs(got - ref) <= 4 * bound)


def test_library_operators_with_the_inflow_on_a_horn():
    xyz, EToV, tag, _ = W.horn_in_room(m1=1, room_length=0.03, room_half=0.03, growth=1.8,
                                       horn_length=0.1, aspect=3.0, behind=0.01)
    geom = Geometry(ReferenceElement(2), xyz, EToV)
    bc_id = np.where(tag < 0, 0, tag)
    modes = {W.HORN_OUTER: CHARACTERISTIC, W.HORN_WALL: SLIP_WALL, W.HORN_MOUTHPIECE: INFLOW_PULSE}
    q = W.gaussian_pulse_state(geom.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, 0.02,
                               center=(0.1, 0.0, 0.0))
    t = 1e-4
    ref = MD.ModalSolver(geom, GAS, bc_id=bc_id, bc_mode=modes, inflow=(0.1, 3000.0)).rhs_nodal(q, t)
    got, bound = _kernel_rhs(B.modal_operators(2), geom, EToV, q, bc_id, modes, t, (0.1, 3000.0))
    # both sides' rounding: the emulation's sums, and the oracle's own (its
    # conversions between nodal values and coefficients, condition <= 16,
    # add rounding of the same order); measured <= 2.5 bounds
    assert np.all(np.abs(got - ref) <= 4 * bound)
    # the bound is tight where it matters: within 1e-11 of the result's scale
    # for density and energy, whose fluxes carry no base pressure
    scale = np.abs(ref).max(axis=(0, 2))
    assert np.all(np.abs(got - ref).max(axis=(0, 2))[[0, 4]] < 1e-11 * scale[[0, 4]])


def test_operator_identities():
    """Exact properties whatever the quadrature: the volume weights of a
    constant flux vanish (sum_q Sv_a[n][q] = d(1)/dr_a terms: the integral of
    grad(phi) over the element is the boundary integral of phi), and the
    face interpolation reproduces constants."""
    for p in (1, 2, 3):
        ops = B.modal_operators(p)
        np.testing.assert_allclose(ops["Ifn"].sum(axis=3), 1.0, atol=1e-13)
        np.testing.assert_allclose(ops["Iq"].sum(axis=1), 1.0, atol=1e-13)
        # int grad(phi) dV = sum_f int phi n dA: on the reference element,
        # sum_q Sv_a[:, q] = sum_f (n_f)_a (reference face areas) sum_q Sf_f[:, q]
        nref = np.array([[0, 0, -1], [0, -1, 0], [1, 1, 1], [-1, 0, 0]], float)   # area-weighted normals / 2
        lhs = ops["Sv"].sum(axis=2)                                            # [3, Np]
        rhs = np.einsum("fa,fn->an", nref, ops["Sf"][:, 0].sum(axis=2))
        np.testing.assert_allclose(lhs, rhs, atol=1e-12)
