"""Pins of the oracle of the paper's own discretisation (oracle/modal_dg.py:
orthonormal basis, Gauss quadrature of degrees 2p and 2p+1, Heun's RK2).

Each test checks it against something other than itself: exact monomial
integrals, orthonormality, free-stream preservation, discrete conservation,
the nodal oracle's strong form where the two discretisations coincide
exactly, the convergence rate against an exact Euler solution, and Heun's
amplification factor."""
import numpy as np
import pytest

from oracle import modal_dg as MD
from oracle.euler_dg import CHARACTERISTIC, FREESTREAM, INFLOW_PULSE, SLIP_WALL, Gas, Solver
from oracle.geometry import Geometry
from oracle.reference_element import (ReferenceElement, exponents2, exponents3, tet_monomial_integral,
                                      tri_monomial_integral, vandermonde3)
from paper_1710_03887_gb300 import workloads as W


@pytest.mark.parametrize("degree", [2, 3, 4, 6, 7, 8, 9])
def test_rules_integrate_monomials_exactly(degree):
    r, s, t, w = MD.tet_rule(degree)
    for a, b, c in exponents3(degree):
        assert abs(w @ (r ** a * s ** b * t ** c) - float(tet_monomial_integral(a, b, c))) < 1e-13
    u, v, wf = MD.tri_rule(degree)
    for a, b in exponents2(degree):
        assert abs(wf @ (u ** a * v ** b) - float(tri_monomial_integral(a, b))) < 1e-13
    # n = degree // 2 + 1 points per direction: one degree more is not exact in general
    n = degree // 2 + 1
    assert len(w) == n ** 3 and len(wf) == n ** 2
    top = 2 * n
    errs = [abs(w @ (r ** a * s ** b * t ** c) - float(tet_monomial_integral(a, b, c)))
            for a, b, c in exponents3(top) if a + b + c == top]
    assert max(errs) > 1e-8


def test_face_points_lie_on_their_faces():
    u, v, _ = MD.tri_rule(5)
    planes = [lambda x: x[:, 2] + 1, lambda x: x[:, 1] + 1, lambda x: x.sum(axis=1) + 1,
              lambda x: x[:, 0] + 1]
    for f in range(4):
        x = MD.face_points(f, u, v)
        assert np.abs(planes[f](x)).max() < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_basis_is_orthonormal(p):
    T = MD.orthonormal_coefficients(p)
    r, s, t, w = MD.tet_rule(2 * p)
    Phi = vandermonde3(p, r, s, t) @ T
    np.testing.assert_allclose(Phi.T @ (w[:, None] * Phi), np.eye(len(exponents3(p))), atol=1e-11)


@pytest.mark.parametrize("mode", [FREESTREAM, CHARACTERISTIC, SLIP_WALL, INFLOW_PULSE])
def test_free_stream_preservation(mode):
    gas = Gas(1.4, 1.4, 1.0)
    xyz, EToV = W.kuhn_cube(3, jitter=0.15, seed=2)
    geom = Geometry(ReferenceElement(2), xyz, EToV)
    S = MD.ModalSolver(geom, gas, bc_mode={0: mode})
    q = W.uniform_state(geom.K, geom.ref.Np, 1.4, (0, 0, 0), 1.0, 1.4)
    r = S.rhs_nodal(q, 0.0)
    assert np.abs(r).max() < 1e-12 * np.abs(geom.Fscale).max()


def test_discrete_conservation_periodic_and_ledger():
    gas = Gas(1.4, 1.4, 1.0)
    ref = ReferenceElement(2)
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=5)
    # periodic box, with the lattice's vertex lists and shuffled ones (both
    # sides of a face must integrate over one point set in every orientation)
    for E in (EToV, W.shuffle_vertices(xyz, EToV, seed=6)):
        geom = Geometry(ref, xyz, E, period=(2.0, 2.0, 2.0))
        S, N = MD.ModalSolver(geom, gas), Solver(geom, gas)
        q = W.random_smooth_state(geom.x, 1.4, 1.4, 1.0, 0.1, seed=2)
        t0 = N.totals(q)
        q2, _, led = S.run(q, 0.5 * N.stable_dt(q), 20)
        np.testing.assert_allclose(N.totals(q2), t0, rtol=0, atol=1e-13 * np.abs(t0).max())
        assert np.all(led == 0.0)
    geom = Geometry(ref, xyz, EToV)
    S, N = MD.ModalSolver(geom, gas), Solver(geom, gas)
    q = W.gaussian_pulse_state(geom.x, 1.4, 1.4, 1.0, 0.2, 0.6)
    t0 = N.totals(q)
    q2, _, led = S.run(q, 0.5 * N.stable_dt(q), 40)
    assert np.abs(led).max() > 1e-4
    assert np.abs(N.totals(q2) - t0 + led).max() <= 1e-13 * np.abs(t0).max()


def _density_wave(x, gas, t, u0):
    rho = 1.0 + 0.2 * np.sin(np.pi * (x[..., 0] + x[..., 1] - t * (u0[0] + u0[1])))
    q = np.empty((x.shape[0], 5, x.shape[1]))
    q[:, 0] = rho
    for d in range(3):
        q[:, 1 + d] = rho * u0[d]
    q[:, 4] = 1.0 / (gas.gamma - 1) + 0.5 * rho * float(np.dot(u0, u0))
    return q


@pytest.mark.parametrize("p", [1, 2, 3])
def test_equals_the_nodal_strong_form_where_both_are_exact(p):
    """A density wave at uniform velocity and pressure, interpolated at the
    nodes, is continuous across faces (zero LLF jumps) and its Euler flux is
    linear in the state, so the flux interpolant is exact and both Gauss
    rules integrate exactly: the weak form of Eq. 10 then equals the nodal
    strong form term by term, on a jittered periodic mesh, with the lattice's
    vertex lists and with shuffled ones (every correspondence between the
    two sides' face vertices, so the two sides' Gauss points must be the
    same physical points whatever the rule's orientation)."""
    gas = Gas(1.4, 1.0, 1.0)
    xyz, EToV = W.kuhn_cube(3, jitter=0.12, seed=p)
    for E in (EToV, W.shuffle_vertices(xyz, EToV, seed=p)):
        geom = Geometry(ReferenceElement(p), xyz, E, period=(2.0, 2.0, 2.0))
        q = _density_wave(geom.x, gas, 0.0, np.array([0.5, 0.3, 0.2]))
        rm = MD.ModalSolver(geom, gas).rhs_nodal(q)
        rn = Solver(geom, gas).rhs(q)
        scale = np.abs(rn).max(axis=(0, 2))
        assert np.all(np.abs(rm - rn).max(axis=(0, 2)) <= 1e-11 * scale)


def test_second_order_convergence_at_p1():
    """The paper's configuration (linear basis, RK2): the density wave's L2
    error falls at rate 2 under refinement at fixed CFL."""
    gas = Gas(1.4, 1.0, 1.0)
    u0 = np.array([0.5, 0.3, 0.2])
    ref = ReferenceElement(1)
    errs, hs = [], []
    T = 0.2
    for n in (2, 4, 8):
        xyz, EToV = W.kuhn_cube(n)
        geom = Geometry(ref, xyz, EToV, period=(2.0, 2.0, 2.0))
        S = MD.ModalSolver(geom, gas)
        q = _density_wave(geom.x, gas, 0.0, u0)
        nst = int(np.ceil(T / Solver(geom, gas).stable_dt(q, 0.3)))
        q, _, _ = S.run(q, T / nst, nst)
        d = q[:, 0] - _density_wave(geom.x, gas, T, u0)[:, 0]
        errs.append(np.sqrt(np.einsum("k,ij,ki,kj->", geom.J, ref.M, d, d)))
        hs.append(2.0 / n)
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert rates[-1] > 1.8, (errs, rates)


def test_heun_amplification_on_a_linear_problem():
    """With f(c) = z c (and a constant ledger rate) one step multiplies by
    1 + z + z^2/2, the amplification factor of every second-order two-stage
    Runge-Kutta method with Heun's weights, and the ledger gains dt times
    the mean of the two stage rates."""
    class Linear(MD.ModalSolver):
        def __init__(self, z):
            self.z = z

        def rhs(self, c, t=0.0):
            return self.z * c, np.full(5, t)

    for z in (-0.3, 0.7, -1.9):
        S = Linear(z)
        c, led = S.step(np.ones((1, 5, 1)), 2.0, 1.0, np.zeros(5))
        assert np.allclose(c, 1 + z + z * z / 2, rtol=1e-15)
        assert np.allclose(led, 0.5 * (2.0 + 3.0))      # stage rates at t and t + dt
