"""The paper's own discretisation of Eq. 10 (test infrastructure, float64).

Only tests/, the smoke check and the bench's CPU legs may use this module; the
library's CUDA path never does.

Appendix A: on each element the solution is U = sum_i c_i phi_i in a basis
orthonormal in L2 (Eq. 11), which makes the mass matrix of Eq. 10 a
multiple of the identity; Eq. 10 with v = phi_i in turn gives the ODE system
dc/dt = f(c) (Eq. 12), whose volume integral is computed by a Gauss rule of
degree 2p and whose surface integral by one of degree 2p+1. Section 1.1
advances Eq. 12 with a second-order Runge-Kutta method and the local
Lax-Friedrichs flux. Written out here directly and slowly:

* basis: the monomials r^a s^b t^c (a+b+c <= p) made orthonormal on the
  reference tetrahedron through the L D L^T factors of their exact Gram
  matrix (rational arithmetic on exact monomial integrals); on the affine element
  phi_i(x) = phihat_i(r(x)), so the physical mass matrix is J I and
      J dc_i/dt = int grad(phi_i) . F(U) dx - sum_faces int phi_i F*(U-, U+, n) dA;
* quadrature: collapsed-coordinate (Duffy) products of Gauss-Jacobi rules
  with n = floor(d/2) + 1 points per direction, exact to degree 2n - 1 >= d
  (d = 2p for the volume, 2p + 1 for the faces). Tetrahedron:
      r = (1+a)(1-b)(1-c)/4 - 1,  s = (1+b)(1-c)/2 - 1,  t = c,
      dr ds dt = (1-b)(1-c)^2/8 da db dc
  (a: Gauss-Legendre, b: Gauss-Jacobi (1,0), c: Gauss-Jacobi (2,0)).
  Triangle (-1,-1), (1,-1), (-1,1): u = (1+a)(1-b)/2 - 1, v = b,
  du dv = (1-b)/2 da db; face f of the tetrahedron is the image of the
  triangle under its vertex triple (1,2,3), (1,2,4), (2,3,4), (1,3,4) with
  barycentric weights (-(u+v)/2, (1+u)/2, (1+v)/2);
* traces: one set of quadrature points per face, so that both elements
  integrate the same flux (the collapsed triangle rule is not symmetric
  under the face's vertex permutations): the rule of the element with the
  lower index, mapped through its own face; each side evaluates its own
  expansion and the neighbour's at those physical points (mapped into the
  respective reference coordinates); on outer faces the element's own rule
  and the ghost states of the nodal oracle (oracle/euler_dg.py) at its
  points;
* time: Heun's method, c1 = c + dt f(c, t), c_next = (c + c1 + dt f(c1, t + dt)) / 2;
  the boundary-flux ledger (the F* integral over outer faces) by the same
  two stages.

Parity status: pinned (tests/test_oracle_modal.py): exactness of both rules
on monomials, orthonormality of the basis, free-stream preservation,
discrete conservation (periodic and with the ledger, also with shuffled
vertex lists so that every face orientation occurs), reduction to the
nodal strong form where both are exact (continuous fields with a flux that
is polynomial in the state), second-order convergence at p = 1, and Heun's
amplification factor on a linear problem; planted mistakes fail them
(tests/test_oracle_pins_catch_mistakes.py).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
from scipy.special import roots_jacobi

from .euler_dg import GHOSTS, INFLOW_PULSE, LEARNED, euler_fluxes, ghost_inflow, llf_flux
from .reference_element import exponents3, tet_monomial_integral, vandermonde3

FACE_VERTS = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))
REF_VERTS = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])


def gauss_jacobi(n, alpha):
    """n-point Gauss rule for the weight (1 - x)^alpha on [-1, 1]."""
    x, w = roots_jacobi(n, alpha, 0.0)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def tet_rule(degree):
    """Collapsed Gauss rule on the reference tetrahedron, exact to ``degree``:
    points (r, s, t) and weights, (degree // 2 + 1)^3 of them."""
    n = degree // 2 + 1
    a, wa = gauss_jacobi(n, 0.0)
    b, wb = gauss_jacobi(n, 1.0)
    c, wc = gauss_jacobi(n, 2.0)
    A, Bb, C = np.meshgrid(a, b, c, indexing="ij")
    W = wa[:, None, None] * wb[None, :, None] * wc[None, None, :] / 8.0
    r = (1 + A) * (1 - Bb) * (1 - C) / 4 - 1
    s = (1 + Bb) * (1 - C) / 2 - 1
    return r.ravel(), s.ravel(), C.ravel(), W.ravel()


def tri_rule(degree):
    """Collapsed Gauss rule on the triangle (-1,-1), (1,-1), (-1,1), exact to
    ``degree``: points (u, v) and weights."""
    n = degree // 2 + 1
    a, wa = gauss_jacobi(n, 0.0)
    b, wb = gauss_jacobi(n, 1.0)
    A, Bb = np.meshgrid(a, b, indexing="ij")
    return ((1 + A) * (1 - Bb) / 2 - 1).ravel(), Bb.ravel(), (wa[:, None] * wb[None, :] / 2).ravel()


def face_points(f, u, v):
    """Reference-tetrahedron points of face f at triangle coordinates (u, v)."""
    lam = np.stack([-(u + v) / 2, (1 + u) / 2, (1 + v) / 2], axis=1)
    return lam @ REF_VERTS[list(FACE_VERTS[f])]


def orthonormal_coefficients(p):
    """T with phi = m T orthonormal on the reference tetrahedron, m the
    monomials of exponents3(p): the exact Gram matrix G of the monomials is
    factored G = L D L^T in rational arithmetic (L unit lower triangular),
    so phi = m L^-T D^-1/2; only the final square roots and the rounding to
    float64 are inexact."""
    ex = exponents3(p)
    n = len(ex)
    G = [[tet_monomial_integral(a1 + a2, b1 + b2, c1 + c2) for a2, b2, c2 in ex] for a1, b1, c1 in ex]
    L = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    D = [Fraction(0)] * n
    for j in range(n):
        D[j] = G[j][j] - sum(L[j][k] * L[j][k] * D[k] for k in range(j))
        for i in range(j + 1, n):
            L[i][j] = (G[i][j] - sum(L[i][k] * L[j][k] * D[k] for k in range(j))) / D[j]
    # Linv = L^-1 (unit lower triangular), by forward substitution
    Linv = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    for i in range(n):
        for j in range(i):
            Linv[i][j] = -sum(L[i][k] * Linv[k][j] for k in range(j, i))
    return np.array([[float(Linv[i][j]) / np.sqrt(float(D[i])) for i in range(n)] for j in range(n)])


class ModalSolver:
    """Eq. 10 in the orthonormal basis with Gauss quadrature, Heun in time.

    ``geom``: oracle Geometry; ``bc_id``/``bc_mode`` as in euler_dg.Solver
    (every mode but the learned closure); ``inflow`` = (A, alpha) of the
    mouthpiece pulse. States are exchanged as nodal values at the nodal
    oracle's interpolation nodes (the modal coefficients of the interpolant
    inside)."""

    def __init__(self, geom, gas, bc_id=None, bc_mode=None, inflow=(0.05, 565.0)):
        g, ref = geom, geom.ref
        p = ref.p
        self.g, self.ref, self.gas, self.inflow = g, ref, gas, inflow
        K = g.K
        self.T = orthonormal_coefficients(p)

        def phi(pts, d=None):
            flat = pts.reshape(-1, 3)
            out = vandermonde3(p, flat[:, 0], flat[:, 1], flat[:, 2], d) @ self.T
            return out.reshape(pts.shape[:-1] + (out.shape[1],))

        rq, sq, tq, self.wq = tet_rule(2 * p)
        vol = np.stack([rq, sq, tq], axis=1)
        self.Phi_q = phi(vol)                                            # [Nq, Np]
        self.dPhi_q = np.stack([phi(vol, d) for d in "rst"])             # [3, Nq, Np]
        u, v, self.wf = tri_rule(2 * p + 1)
        fpts = np.stack([face_points(f, u, v) for f in range(4)])        # [4, Nfq, 3]
        self.Phi_f = np.stack([phi(fpts[f]) for f in range(4)])          # [4, Nfq, Np]
        nodes = np.stack([ref.r, ref.s, ref.t], axis=1)
        self.Phi_nodes = phi(nodes)                                      # [Np, Np]
        self.Phi_nodes_inv = np.linalg.inv(self.Phi_nodes)
        # affine maps: x = v1 + Jm (r + 1)
        assert np.allclose(nodes[0], -1.0)                               # node 0 is vertex 1
        v1 = g.x[:, 0, :]
        Jm = np.linalg.inv(g.drdx)                                       # [K, 3, 3] dx/dr
        own_std = v1[:, None, None, :] + np.einsum("kij,fqj->kfqi", Jm, fpts + 1.0)   # [K, 4, Nfq, 3]
        verts = v1[:, None, :] + np.einsum("kij,cj->kci", Jm, REF_VERTS + 1.0)      # [K, 4, 3]
        fc = np.stack([verts[:, list(FACE_VERTS[f])].mean(axis=1) for f in range(4)], axis=1)
        # one point set per face: the rule of the element with the lower
        # index, seen by the other through the shared physical points (the
        # offset between the two faces' centroids is nonzero only across a
        # periodic seam)
        e2, f2 = g.EToE, g.EToF
        shift = fc - fc[e2, f2]                                          # [K, 4, 3]
        mine = (np.arange(K)[:, None] <= e2) | g.boundary
        X = np.where(mine[:, :, None, None], own_std, own_std[e2, f2] + shift[:, :, None, :])
        r_own = -1.0 + np.einsum("kij,kfqj->kfqi", g.drdx, X - v1[:, None, None, :])
        r_nbr = -1.0 + np.einsum("kfij,kfqj->kfqi", g.drdx[e2],
                                 X - shift[:, :, None, :] - v1[e2][:, :, None, :])
        self.Phi_own = phi(r_own)                                        # [K, 4, Nfq, Np]
        self.Phi_nbr = phi(r_nbr)
        bnd = g.boundary
        self.bc_id = np.zeros((K, 4), dtype=np.int64) if bc_id is None else np.asarray(bc_id)
        self.bc_mode = {0: 1} if bc_mode is None else dict(bc_mode)
        self.groups = []
        if np.any(bnd):
            bidx = np.nonzero(bnd)
            for ident in np.unique(self.bc_id[bidx]):
                mode = self.bc_mode[int(ident)]
                if mode == LEARNED:
                    raise ValueError("the modal oracle has no learned closure")
                self.groups.append((mode, tuple(ix[self.bc_id[bidx] == ident] for ix in bidx)))

    # -- nodal values <-> coefficients of the interpolant
    def to_coefficients(self, q):
        return np.einsum("ij,kvj->kvi", self.Phi_nodes_inv, q)

    def to_nodal(self, c):
        return np.einsum("ij,kvj->kvi", self.Phi_nodes, c)

    # -- Eq. 10 / Eq. 12
    def rhs(self, c, t=0.0):
        """(dc/dt, rate of the boundary-flux ledger) at coefficients c, time t."""
        g, gas = self.g, self.gas
        gam = gas.gamma
        Uq = np.einsum("qj,kvj->kqv", self.Phi_q, c)                     # [K, Nq, 5]
        flux = np.stack(euler_fluxes(Uq, gam), axis=1)                   # [K, 3 (x,y,z), Nq, 5]
        # grad phi_i in x: sum_a dphi_i/dr_a dr_a/dx_d
        gphi = np.einsum("aqi,kad->kdqi", self.dPhi_q, g.drdx)           # [K, 3, Nq, Np]
        vol = np.einsum("q,kdqi,kdqv->kvi", self.wq, gphi, flux) * g.J[:, None, None]
        Um = np.einsum("kfqj,kvj->kfqv", self.Phi_own, c)                # [K, 4, Nfq, 5]
        Up = np.einsum("kfqj,kfvj->kfqv", self.Phi_nbr, c[g.EToE])
        n = np.broadcast_to(g.nrm[:, :, None, :], Um.shape[:3] + (3,))
        for mode, sel in self.groups:
            if mode == INFLOW_PULSE:
                Up[sel] = ghost_inflow(Um[sel], n[sel], gas, t, *self.inflow)
            else:
                Up[sel] = GHOSTS[mode](Um[sel], n[sel], gas)
        fstar = llf_flux(Um, Up, n, gam)                                 # [K, 4, Nfq, 5]
        surf = np.einsum("kf,q,kfqi,kfqv->kvi", g.sJ, self.wf, self.Phi_own, fstar)
        ledger = np.einsum("kf,q,kfqv->v", g.sJ * g.boundary, self.wf, fstar)
        return (vol - surf) / g.J[:, None, None], ledger

    def step(self, c, t, dt, ledger):
        """Heun's method on Eq. 12 and on the ledger."""
        k1, b1 = self.rhs(c, t)
        c1 = c + dt * k1
        k2, b2 = self.rhs(c1, t + dt)
        return 0.5 * (c + c1 + dt * k2), ledger + 0.5 * dt * (b1 + b2)

    def run(self, q, dt, nsteps, t=0.0):
        """nsteps steps from nodal values q: (nodal values, t, ledger)."""
        c = self.to_coefficients(q)
        ledger = np.zeros(5)
        for _ in range(nsteps):
            c, ledger = self.step(c, t, dt, ledger)
            t += dt
        return self.to_nodal(c), t, ledger

    def rhs_nodal(self, q, t=0.0):
        """dq/dt of the nodal values (the interpolant's time derivative)."""
        dc, _ = self.rhs(self.to_coefficients(q), t)
        return self.to_nodal(dc)
