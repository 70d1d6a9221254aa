"""Element geometry and connectivity of the oracle (test infrastructure, float64).

The paper partitions the domain into non-overlapping elements (Appendix A,
Eq. 9) and couples neighbours only through the flux on their shared face
(the surface term of Eq. 10). For straight-sided tetrahedra everything
needed is a property of the affine map

    x(r,s,t) = ( -(1+r+s+t) v1 + (1+r) v2 + (1+s) v3 + (1+t) v4 ) / 2,

computed here directly from its definition:

* J = det(dx/d(r,s,t)) = element volume / (4/3),
* (rx .. tz) = entries of the inverse Jacobian matrix,
* outward unit normal and area of each face from the cross product of two
  edges, sJ = area / 2 (the face's parameter triangle has area 2),
  Fscale = sJ / J.

Connectivity is found by geometry only: two faces are neighbours when their
centroids coincide (optionally modulo a periodic box), and the nodes of a
shared face are paired by coordinate match. This is deliberately unlike a
combinatorial vertex-triple matcher.

Parity status: pinned (tests/test_oracle_geometry.py: closed-surface identity
sum sJ n = 0, volumes, opposite normals of neighbours, node pairing).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .reference_element import ReferenceElement


class Geometry:
    """Geometric factors and connectivity of a straight-sided tetrahedral mesh.

    ``period``: None, or the box edge length vector (Lx, Ly, Lz) of a
    periodic box whose lower corner is ``box_lo``; faces on opposite box sides
    are then neighbours.
    """

    def __init__(self, ref: ReferenceElement, xyz, EToV, period=None,
                 box_lo=(-1.0, -1.0, -1.0)):
        self.ref = ref
        xyz = np.asarray(xyz, dtype=np.float64)
        EToV = np.asarray(EToV, dtype=np.int64)
        K = EToV.shape[0]
        self.K = K
        v = xyz[EToV]                                          # [K, 4, 3]
        self.verts = v
        # node coordinates from the affine map
        r, s, t = ref.r, ref.s, ref.t
        w = 0.5 * np.stack([-(1 + r + s + t), 1 + r, 1 + s, 1 + t], axis=0)  # [4, Np]
        self.x = np.einsum("an,kai->kni", w, v)               # [K, Np, 3]
        # Jacobian matrix columns dx/dr, dx/ds, dx/dt
        Jm = 0.5 * np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0],
                             v[:, 3] - v[:, 0]], axis=2)       # [K, 3(x), 3(r)]
        self.J = np.linalg.det(Jm)
        if np.any(self.J <= 0):
            raise ValueError("non-positive element Jacobian")
        inv = np.linalg.inv(Jm)                                # [K, 3(r), 3(x)]
        self.drdx = inv                                        # drdx[k, a, b] = d r_a / d x_b
        # faces: vertex triples in the reference face order
        fv = [(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)]
        opp = [3, 2, 0, 1]
        nrm = np.zeros((K, 4, 3))
        area = np.zeros((K, 4))
        for f, (a, b, c) in enumerate(fv):
            cr = np.cross(v[:, b] - v[:, a], v[:, c] - v[:, a])
            ar = 0.5 * np.linalg.norm(cr, axis=1)
            n = cr / (2.0 * ar)[:, None]
            # orient outward: away from the opposite vertex
            sgn = np.sign(np.einsum("ki,ki->k", n, v[:, a] - v[:, opp[f]]))
            nrm[:, f] = n * sgn[:, None]
            area[:, f] = ar
        self.nrm = nrm
        self.area = area
        self.sJ = area / 2.0
        self.Fscale = self.sJ / self.J[:, None]
        self.volume = self.J * 4.0 / 3.0
        self._connect(period, np.asarray(box_lo, dtype=np.float64))

    def _wrap(self, pts, period, lo):
        if period is None:
            return pts
        L = np.asarray(period, dtype=np.float64)
        rel = (pts - lo) / L
        rel = rel - np.floor(rel + 1e-9)
        return lo + rel * L

    def _connect(self, period, lo):
        ref, K = self.ref, self.K
        Fm = ref.Fmask
        # face centroids
        fc = np.stack([self.x[:, Fm[f]].mean(axis=1) for f in range(4)], axis=1)  # [K,4,3]
        pts = self._wrap(fc.reshape(-1, 3), period, lo)
        h = np.min(np.cbrt(self.volume))
        tol = 1e-6 * h
        tree = cKDTree(pts)
        pairs = tree.query_pairs(tol, output_type="ndarray")
        EToE = np.tile(np.arange(K)[:, None], (1, 4))
        EToF = np.tile(np.arange(4)[None, :], (K, 1))
        seen = np.zeros(4 * K, dtype=np.int64)
        for a, b in pairs:
            seen[a] += 1
            seen[b] += 1
            EToE[a // 4, a % 4], EToF[a // 4, a % 4] = b // 4, b % 4
            EToE[b // 4, b % 4], EToF[b // 4, b % 4] = a // 4, a % 4
        if np.any(seen > 1):
            raise ValueError("a face matches more than one other face")
        self.EToE, self.EToF = EToE, EToF
        self.boundary = seen == 0                              # [4K] flags
        self.boundary = self.boundary.reshape(K, 4)
        # pair face nodes by coordinates: vmapP[k, f, m] = flat node index
        Nfp = ref.Nfp
        vmapP = np.zeros((K, 4, Nfp), dtype=np.int64)
        xf = self._wrap(self.x.reshape(-1, 3), period, lo).reshape(K, -1, 3)
        for k in range(K):
            for f in range(4):
                own = xf[k, Fm[f]]
                if self.boundary[k, f]:
                    vmapP[k, f] = k * ref.Np + Fm[f]
                    continue
                k2, f2 = EToE[k, f], EToF[k, f]
                other = xf[k2, Fm[f2]]
                d = np.linalg.norm(own[:, None, :] - other[None, :, :], axis=2)
                j = np.argmin(d, axis=1)
                if np.any(d[np.arange(Nfp), j] > tol) or len(set(j)) != Nfp:
                    raise ValueError("face nodes do not pair up")
                vmapP[k, f] = k2 * ref.Np + Fm[f2][j]
        self.vmapP = vmapP
        self.vmapM = (np.arange(K)[:, None, None] * ref.Np + Fm[None, :, :])

    def metric(self):
        """(rx, ry, rz, sx, ..., tz) as a [K, 3, 3] array m[k, a, b] = d r_a / d x_b."""
        return self.drdx


def inscribed_radius(geom):
    """r_in = 3 V / (sum of face areas), per element."""
    return 3.0 * geom.volume / geom.area.sum(axis=1)
