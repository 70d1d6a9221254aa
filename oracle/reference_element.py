"""Reference tetrahedron of the oracle (test infrastructure, float64).

The paper expands the solution on each element in a polynomial basis of
degree p (Appendix A, Eq. 11) and obtains the semi-discrete system from the
element-wise weak form (Eq. 10). The solver under test is nodal: the unknowns
are point values at Np = (p+1)(p+2)(p+3)/6 interpolation nodes. This module
builds, by their definitions and nothing cleverer:

* the node set: Warburton's warp-and-blend construction with blending
  exponent zero (nodes on every edge are the 1D Legendre-Gauss-Lobatto points);
* the Lagrange basis l_i of those nodes, written through the monomials
  r^a s^b t^c (a+b+c <= p) and the Vandermonde matrix;
* D_r, D_s, D_t: D_r[i, j] = dl_j/dr at node i;
* the mass matrix M[i, j] = integral of l_i l_j over the tetrahedron, from
  exact monomial integrals;
* faces, their node lists, the face mass matrices (integrals over the face in
  its two parameter coordinates) and LIFT = M^-1 E.

All matrices are formed in exact rational arithmetic (Python Fractions)
from the float64 node coordinates and rounded to float64 once at the end.

Reference tetrahedron: vertices v1 = (-1,-1,-1), v2 = (1,-1,-1),
v3 = (-1,1,-1), v4 = (-1,-1,1). Faces in order: 1: t = -1, 2: s = -1,
3: r+s+t = -1, 4: r = -1. Face parameters: (r,s), (r,t), (s,t), (s,t).

Node order: lattice index (i, j, k) with i counting along r, j along s, k
along t, i+j+k <= p; k outermost, i innermost.

Parity status: pinned (tests/test_oracle_reference.py: LGL edge nodes, exact
differentiation of polynomials, integrals of monomials, symmetry of the node
set, face-mass sums).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import comb, factorial

import numpy as np

# ----------------------------------------------------------------- 1D points

def lgl_points(p):
    """Legendre-Gauss-Lobatto points on [-1, 1]: +-1 and the roots of P_p'."""
    if p == 1:
        return np.array([-1.0, 1.0])
    inner = np.polynomial.legendre.Legendre.basis(p).deriv().roots()
    x = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    return x


def warp_factor(p, x):
    """phi(x) = w(x) / (1 - x^2), w = interpolant of (LGL - equispaced).

    w is the degree-p polynomial through the p+1 equispaced points of [-1,1]
    whose values are the displacements that move each equispaced point onto
    the matching LGL point. Both end displacements are zero, so w has the
    factor (1 - x^2); phi is the quotient, evaluated through the interior
    Lagrange factors so it stays finite at x = +-1.
    """
    x = np.asarray(x, dtype=np.float64)
    xe = np.linspace(-1.0, 1.0, p + 1)
    disp = lgl_points(p) - xe
    phi = np.zeros_like(x)
    for i in range(1, p):
        term = np.full_like(x, disp[i] / (1.0 - xe[i] ** 2))
        for j in range(1, p):
            if j != i:
                term = term * (x - xe[j]) / (xe[i] - xe[j])
        phi += term
    return phi


# --------------------------------------------------------------- node set

def lattice(p):
    """Lattice indices (i, j, k), i+j+k <= p, in the node order."""
    out = []
    for k in range(p + 1):
        for j in range(p + 1 - k):
            for i in range(p + 1 - k - j):
                out.append((i, j, k))
    return np.array(out, dtype=np.int64)


def _equilateral_vertices():
    s3, s6 = np.sqrt(3.0), np.sqrt(6.0)
    return np.array([[-1.0, -1.0 / s3, -1.0 / s6],
                     [1.0, -1.0 / s3, -1.0 / s6],
                     [0.0, 2.0 / s3, -1.0 / s6],
                     [0.0, 0.0, 3.0 / s6]])


@lru_cache(maxsize=None)
def nodes(p):
    """Warp-and-blend nodes (blending exponent 0) as (r, s, t), each [Np]."""
    L = lattice(p)
    lam = np.stack([p - L.sum(axis=1), L[:, 0], L[:, 1], L[:, 2]],
                   axis=1).astype(np.float64) / p          # barycentrics of v1..v4
    X = _equilateral_vertices()
    pos = lam @ X
    faces = [(0, 1, 2, 3), (0, 1, 3, 2), (1, 2, 3, 0), (0, 2, 3, 1)]  # 3 face vertices + opposite
    tol = 1e-10
    shift = np.zeros_like(pos)
    on_edge = (lam < tol).sum(axis=1) == 2
    for a, b, c, o in faces:
        warp = np.zeros_like(pos)
        for u, v in ((a, b), (b, c), (c, a)):
            # edge u -> v: displacement along the edge, zero off the edge's face
            amount = 4.0 * lam[:, u] * lam[:, v] * warp_factor(p, lam[:, v] - lam[:, u])
            warp += amount[:, None] * (X[v] - X[u])[None, :] / 2.0
        num = lam[:, a] * lam[:, b] * lam[:, c]
        den = ((lam[:, a] + 0.5 * lam[:, o]) * (lam[:, b] + 0.5 * lam[:, o])
               * (lam[:, c] + 0.5 * lam[:, o]))
        blend = np.where(den > tol, num / np.where(den > tol, den, 1.0), 0.0)
        shift += blend[:, None] * warp
        # a node on an edge of this face takes the face warp itself, which is
        # the 1D LGL displacement along that edge
        sel = on_edge & (lam[:, o] < tol)
        shift[sel] = warp[sel]
    pos = pos + shift
    # back to reference coordinates through barycentrics of the equilateral tet
    A = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    mu = np.linalg.solve(A, (pos - X[0]).T).T              # (lam2, lam3, lam4)
    r = -1.0 + 2.0 * mu[:, 0]
    s = -1.0 + 2.0 * mu[:, 1]
    t = -1.0 + 2.0 * mu[:, 2]
    return r, s, t


def n_nodes(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def n_face_nodes(p):
    return (p + 1) * (p + 2) // 2


# ---------------------------------------------------------- monomial basis

def exponents3(p):
    return [(a, b, c) for a in range(p + 1) for b in range(p + 1 - a)
            for c in range(p + 1 - a - b)]


def exponents2(p):
    return [(a, b) for a in range(p + 1) for b in range(p + 1 - a)]


def vandermonde3(p, r, s, t, d=None):
    """Monomials (or their r/s/t derivative, d in 'rst') at points: [npts, Np]."""
    cols = []
    for a, b, c in exponents3(p):
        if d is None:
            cols.append(r ** a * s ** b * t ** c)
        elif d == "r":
            cols.append(a * r ** max(a - 1, 0) * s ** b * t ** c if a else 0.0 * r)
        elif d == "s":
            cols.append(b * r ** a * s ** max(b - 1, 0) * t ** c if b else 0.0 * r)
        elif d == "t":
            cols.append(c * r ** a * s ** b * t ** max(c - 1, 0) if c else 0.0 * r)
    return np.stack(cols, axis=1)


def vandermonde2(p, u, v):
    return np.stack([u ** a * v ** b for a, b in exponents2(p)], axis=1)


def _shifted_power_integral(exps, dim):
    """Exact integral of prod (2 x_k - 1)^{e_k} over the unit simplex of dimension dim.

    Uses  int x^i y^j (z^k) = i! j! (k!) / (i + j (+ k) + dim)!  on the unit simplex.
    """
    total = Fraction(0)

    def rec(k, powers, coef):
        nonlocal total
        if k == len(exps):
            num = 1
            for q in powers:
                num *= factorial(q)
            total += coef * Fraction(num, factorial(sum(powers) + dim))
            return
        e = exps[k]
        for q in range(e + 1):
            rec(k + 1, powers + [q], coef * comb(e, q) * 2 ** q * (-1) ** (e - q))

    rec(0, [], Fraction(1))
    return total


def tet_monomial_integral(a, b, c):
    """Exact integral of r^a s^b t^c over the reference tetrahedron.

    The map r = 2x - 1 (etc.) takes the unit simplex onto it with Jacobian 8.
    """
    return 8 * _shifted_power_integral([a, b, c], 3)


def tri_monomial_integral(a, b):
    """Exact integral of u^a v^b over the triangle u, v >= -1, u + v <= 0."""
    return 4 * _shifted_power_integral([a, b], 2)


# ------------------------------------------------- exact rational algebra

def _q(x):
    return Fraction(float(x))


def _mat(rows):
    return [list(r) for r in rows]


def _matmul(A, B):
    Bt = list(zip(*B))
    return [[sum((a * b for a, b in zip(row, col)), Fraction(0)) for col in Bt] for row in A]


def _transpose(A):
    return [list(r) for r in zip(*A)]


def _inverse(A):
    """Exact Gauss-Jordan inverse of a square matrix of Fractions."""
    n = len(A)
    W = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for c in range(n):
        piv = next((i for i in range(c, n) if W[i][c] != 0), None)
        if piv is None:
            raise ValueError("singular matrix")
        W[c], W[piv] = W[piv], W[c]
        d = W[c][c]
        W[c] = [x / d for x in W[c]]
        for i in range(n):
            if i != c and W[i][c] != 0:
                f = W[i][c]
                W[i] = [x - f * y for x, y in zip(W[i], W[c])]
    return [row[n:] for row in W]


def _to_float(A):
    return np.array([[float(x) for x in row] for row in A])


def _mono3(ex, r, s, t, d=None):
    """Monomials (or a derivative) at exact points, as Fractions: [npts][Np]."""
    out = []
    for x, y, z in zip(r, s, t):
        row = []
        for a, b, c in ex:
            if d is None:
                row.append(x ** a * y ** b * z ** c)
            elif d == "r":
                row.append(a * x ** (a - 1) * y ** b * z ** c if a else Fraction(0))
            elif d == "s":
                row.append(b * x ** a * y ** (b - 1) * z ** c if b else Fraction(0))
            else:
                row.append(c * x ** a * y ** b * z ** (c - 1) if c else Fraction(0))
        out.append(row)
    return out


# ----------------------------------------------------------------- operators

@lru_cache(maxsize=None)
def _exact_operators(p):
    """All operators in exact rational arithmetic from the float64 nodes."""
    r, s, t = nodes(p)
    R, S, T = [_q(x) for x in r], [_q(x) for x in s], [_q(x) for x in t]
    ex = exponents3(p)
    V = _mono3(ex, R, S, T)
    Vinv = _inverse(V)
    D = [_matmul(_mono3(ex, R, S, T, d), Vinv) for d in "rst"]
    G = [[tet_monomial_integral(a1 + a2, b1 + b2, c1 + c2) for (a2, b2, c2) in ex]
         for (a1, b1, c1) in ex]
    # M[i][j] = int l_i l_j = (Vinv^T G Vinv)[i][j];  M^-1 = V G^-1 V^T
    M = _matmul(_matmul(_transpose(Vinv), G), Vinv)
    Minv = _matmul(_matmul(V, _inverse(G)), _transpose(V))
    tol = 1e-10
    face_sel = [np.abs(t + 1) < tol, np.abs(s + 1) < tol,
                np.abs(r + s + t + 1) < tol, np.abs(r + 1) < tol]
    Fmask = [list(np.nonzero(m)[0]) for m in face_sel]
    par = [(R, S), (R, T), (S, T), (S, T)]
    ex2 = exponents2(p)
    G2 = [[tri_monomial_integral(a1 + a2, b1 + b2) for (a2, b2) in ex2] for (a1, b1) in ex2]
    Np, Nfp = len(R), len(Fmask[0])
    E = [[Fraction(0)] * (4 * Nfp) for _ in range(Np)]
    face_mass = []
    for f in range(4):
        u = [par[f][0][n] for n in Fmask[f]]
        v = [par[f][1][n] for n in Fmask[f]]
        V2inv = _inverse([[x ** a * y ** b for (a, b) in ex2] for x, y in zip(u, v)])
        Mf = _matmul(_matmul(_transpose(V2inv), G2), V2inv)
        face_mass.append(Mf)
        for i, n in enumerate(Fmask[f]):
            for j in range(Nfp):
                E[n][f * Nfp + j] = Mf[i][j]
    LIFT = _matmul(Minv, E)
    return dict(V=V, Vinv=Vinv, D=D, M=M, E=E, LIFT=LIFT, face_mass=face_mass,
                Fmask=np.array(Fmask, dtype=np.int64))


class ReferenceElement:
    """All reference-element operators of order p.

    Built in exact rational arithmetic from the float64 node coordinates
    (the only rounding is the final conversion to float64), so the oracle's
    operators are the exact operators of its node set.
    """

    def __init__(self, p):
        if p < 1:
            raise ValueError("order must be >= 1")
        self.p = p
        self.Np = n_nodes(p)
        self.Nfp = n_face_nodes(p)
        self.r, self.s, self.t = nodes(p)
        X = _exact_operators(p)
        self.V = _to_float(X["V"])
        self.Vinv = _to_float(X["Vinv"])
        self.Dr, self.Ds, self.Dt = (_to_float(d) for d in X["D"])
        self.M = _to_float(X["M"])
        self.E = _to_float(X["E"])
        self.LIFT = _to_float(X["LIFT"])
        self.face_mass = [_to_float(m) for m in X["face_mass"]]
        self.Fmask = X["Fmask"]

    def interp_row(self, r, s, t):
        """Values of the Lagrange basis at reference points: [npts, Np]."""
        r, s, t = (np.atleast_1d(np.asarray(x, dtype=np.float64)) for x in (r, s, t))
        return vandermonde3(self.p, r, s, t) @ self.Vinv
