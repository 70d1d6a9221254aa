"""Pins of the oracle's reference element against closed forms and quadrature."""
import itertools
from pathlib import Path

import numpy as np
import pytest

from oracle.reference_element import ReferenceElement, lgl_points, nodes, tet_monomial_integral

GOLDEN = Path(__file__).parent / "golden"


def _golden_lgl():
    out = {}
    for line in (GOLDEN / "lgl_points.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            vals = line.split()
            out[int(vals[0])] = np.array([float(v) for v in vals[1:]])
    return out


def duffy_quadrature(n=8):
    """Gauss-Legendre on the cube mapped onto the reference tetrahedron."""
    x, w = np.polynomial.legendre.leggauss(n)
    A, B, Cc = np.meshgrid(x, x, x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    r = (1 + A) * (1 - B) * (1 - Cc) / 4 - 1
    s = (1 + B) * (1 - Cc) / 2 - 1
    t = Cc
    jac = (1 - B) * (1 - Cc) ** 2 / 8
    return r.ravel(), s.ravel(), t.ravel(), (W * jac).ravel()


def random_poly(p, rng):
    """Random polynomial of total degree p: (f, df/dr, df/ds, df/dt) callables."""
    terms = [(a, b, c, rng.normal()) for a in range(p + 1) for b in range(p + 1 - a)
             for c in range(p + 1 - a - b)]

    def f(r, s, t):
        return sum(k * r ** a * s ** b * t ** c for a, b, c, k in terms)

    def fr(r, s, t):
        return sum(k * a * r ** max(a - 1, 0) * s ** b * t ** c for a, b, c, k in terms)

    def fs(r, s, t):
        return sum(k * b * r ** a * s ** max(b - 1, 0) * t ** c for a, b, c, k in terms)

    def ft(r, s, t):
        return sum(k * c * r ** a * s ** b * t ** max(c - 1, 0) for a, b, c, k in terms)

    return f, fr, fs, ft


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_lgl_points_closed_form(p):
    np.testing.assert_allclose(lgl_points(p)[1:-1], _golden_lgl()[p], atol=1e-14)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_edges_carry_lgl_points(p):
    r, s, t = nodes(p)
    gold = np.concatenate([[-1.0], _golden_lgl()[p], [1.0]])
    # edge v1-v2 (s = t = -1) and edge v3-v4 (r = -1, s + t = 0)
    e12 = np.sort(r[(np.abs(s + 1) < 1e-12) & (np.abs(t + 1) < 1e-12)])
    np.testing.assert_allclose(e12, gold, atol=1e-14)
    e34 = np.sort(t[(np.abs(r + 1) < 1e-12) & (np.abs(s + t) < 1e-12)])
    np.testing.assert_allclose(e34, gold, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_node_set_invariant_under_vertex_permutations(p):
    r, s, t = nodes(p)
    lam = np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], axis=1)
    key = lambda L: np.array(sorted(map(tuple, np.round(L, 12))))
    base = key(lam)
    for perm in itertools.permutations(range(4)):
        np.testing.assert_array_equal(key(lam[:, perm]), base)
    assert len(r) == (p + 1) * (p + 2) * (p + 3) // 6
    assert np.all(lam > -1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_derivative_matrices_exact_on_polynomials(p):
    R = ReferenceElement(p)
    rng = np.random.default_rng(p)
    for _ in range(3):
        f, fr, fs, ft = random_poly(p, rng)
        u = f(R.r, R.s, R.t)
        np.testing.assert_allclose(R.Dr @ u, fr(R.r, R.s, R.t), atol=1e-11)
        np.testing.assert_allclose(R.Ds @ u, fs(R.r, R.s, R.t), atol=1e-11)
        np.testing.assert_allclose(R.Dt @ u, ft(R.r, R.s, R.t), atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_matrix_against_quadrature(p):
    R = ReferenceElement(p)
    rng = np.random.default_rng(10 + p)
    qr, qs, qt, qw = duffy_quadrature(p + 3)
    for _ in range(3):
        f = random_poly(p, rng)[0]
        g = random_poly(p, rng)[0]
        exact = np.sum(qw * f(qr, qs, qt) * g(qr, qs, qt))
        got = f(R.r, R.s, R.t) @ R.M @ g(R.r, R.s, R.t)
        assert got == pytest.approx(exact, rel=1e-12, abs=1e-12)


def test_monomial_integrals_against_quadrature():
    qr, qs, qt, qw = duffy_quadrature(8)
    assert float(tet_monomial_integral(0, 0, 0)) == pytest.approx(4.0 / 3.0, rel=1e-15)
    for a, b, c in [(1, 0, 0), (0, 2, 1), (3, 1, 2), (2, 2, 2), (0, 0, 5)]:
        ref = np.sum(qw * qr ** a * qs ** b * qt ** c)
        assert float(tet_monomial_integral(a, b, c)) == pytest.approx(ref, rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_summation_by_parts(p):
    """Integration by parts on the reference element, per direction:
    M D_x + (M D_x)^T = sum over faces of n_x * (area ratio) * E_f,
    which ties M, D, the face lists and the face mass matrices together.
    Face 3 (r+s+t=-1) has normal (1,1,1)/sqrt(3) and physical/parameter area
    ratio sqrt(3); faces 1, 2, 4 have normals -t, -s, -r and ratio 1."""
    R = ReferenceElement(p)
    Np, Nfp = R.Np, R.Nfp

    def Ef(f):
        out = np.zeros((Np, Np))
        out[np.ix_(R.Fmask[f], R.Fmask[f])] = R.face_mass[f]
        return out

    E = [Ef(f) for f in range(4)]
    for D, neg in ((R.Dr, 3), (R.Ds, 1), (R.Dt, 0)):
        lhs = R.M @ D + (R.M @ D).T
        np.testing.assert_allclose(lhs, E[2] - E[neg], atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_face_mass_and_lift(p):
    R = ReferenceElement(p)
    for f in range(4):
        assert R.face_mass[f].sum() == pytest.approx(2.0, rel=1e-13)   # parameter area
    # M LIFT = E (definition of LIFT) and LIFT maps face data to volume nodes
    np.testing.assert_allclose(R.M @ R.LIFT, R.E, atol=1e-12)
    # the face node lists are exactly the nodes on each face
    tol = 1e-12
    on = [np.abs(R.t + 1) < tol, np.abs(R.s + 1) < tol, np.abs(R.r + R.s + R.t + 1) < tol,
          np.abs(R.r + 1) < tol]
    for f in range(4):
        assert sorted(R.Fmask[f]) == list(np.nonzero(on[f])[0])
        assert len(R.Fmask[f]) == (p + 1) * (p + 2) // 2


@pytest.mark.parametrize("p", [1, 3])
def test_interpolation_reproduces_polynomials(p):
    R = ReferenceElement(p)
    f = random_poly(p, np.random.default_rng(4))[0]
    pts = np.array([[-0.5, -0.5, -0.5], [-0.9, -0.2, 0.0], [0.1, -0.8, -0.4]])
    row = R.interp_row(pts[:, 0], pts[:, 1], pts[:, 2])
    np.testing.assert_allclose(row @ f(R.r, R.s, R.t), f(*pts.T), atol=1e-12)
