"""Shared set-up of matched oracle / library runs for the tests.

Both sides get the same mesh arrays, boundary tags and initial state (the
state is evaluated at the oracle's node coordinates, which the host-logic
tests show agree with the library's to rounding).
"""
from __future__ import annotations

import numpy as np

from oracle.euler_dg import CHARACTERISTIC, FREESTREAM, SLIP_WALL, Gas, Probes, Solver
from oracle.geometry import Geometry
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import workloads as W

SI = dict(gamma=W.GAMMA, rho0=W.RHO0_SI, p0=W.P0_SI)
SCALED = dict(gamma=1.4, rho0=1.4, p0=1.0)          # the paper's scaling, c0 = 1 (Eq. 3)


def rel_err(a, b):
    """Per conserved variable: max |a - b| / max |b| (q arrays [K, 5, Np])."""
    a = np.asarray(a)
    b = np.asarray(b)
    num = np.abs(a - b).max(axis=(0, 2))
    den = np.abs(b).max(axis=(0, 2))
    return num / np.where(den > 0, den, 1.0)


def state_err(a, b, gas):
    """Per conserved variable: max |a - b| / scale, with scale = max |b| for
    density and energy and rho0 * c0 for the momentum components."""
    num = np.abs(np.asarray(a) - np.asarray(b)).max(axis=(0, 2))
    den = np.abs(np.asarray(b)).max(axis=(0, 2))
    den[1:4] = np.maximum(den[1:4], gas.rho0 * gas.c0)
    return num / den


def direction_tags(xyz, EToV, ref_geom):
    """Boundary ids by outward normal direction: x faces 0, y faces 1, z faces 2."""
    tags = np.full((EToV.shape[0], 4), -1, dtype=np.int8)
    b = ref_geom.boundary
    ax = np.argmax(np.abs(ref_geom.nrm), axis=2)
    tags[b] = ax[b]
    return tags


class Case:
    def __init__(self, p, xyz, EToV, gas=SI, tags=None, modes=None, period=None):
        self.p = p
        self.xyz, self.EToV = xyz, EToV
        self.ref = ReferenceElement(p)
        self.geom = Geometry(self.ref, xyz, EToV, period=period)
        self.gas = Gas(gas["gamma"], gas["rho0"], gas["p0"])
        self.gas_kw = gas
        self.tags = tags
        self.modes = {0: CHARACTERISTIC} if modes is None else modes
        bc_id = None if tags is None else np.where(tags < 0, 0, tags)
        self.oracle = Solver(self.geom, self.gas, bc_id=bc_id, bc_mode=self.modes)
        self.period = period

    def library(self):
        from paper_1710_03887_gb300 import binding as B
        S = B.Solver(self.p, **self.gas_kw)
        vclass = None
        if self.period is not None:
            n = round(np.cbrt(self.EToV.shape[0] / 6))
            vclass = W.periodic_vertex_classes(n)
        S.upload_mesh(self.xyz, self.EToV, face_tag=self.tags, vert_class=vclass)
        for ident, mode in self.modes.items():
            S.set_bc(ident, mode)
        return S

    def pulse(self, amplitude, width=0.15, center=(0.0, 0.0, 0.0)):
        g = self.gas_kw
        return W.gaussian_pulse_state(self.geom.x, g["gamma"], g["rho0"], g["p0"],
                                      amplitude, width, center)

    def smooth(self, amplitude=0.05, seed=0):
        g = self.gas_kw
        return W.random_smooth_state(self.geom.x, g["gamma"], g["rho0"], g["p0"], amplitude, seed)


__all__ = ["Case", "rel_err", "state_err", "direction_tags", "SI", "SCALED", "CHARACTERISTIC", "FREESTREAM",
           "SLIP_WALL", "Probes"]


U32 = 2.0 ** -24          # unit roundoff of float32, round to nearest


def f32_contraction_bound(osol, q, gas, parts=False):
    """Rounding bound of the float32 stage at each node and variable, two parts.

    Arithmetic: (K + 10) u (sum_a |D_a| |F~'_a| + |LIFT| |dF|), the standard
    bound of a K-term float32 dot product (K = 3 Np + 4 Nfp) applied to Eq.
    10's two contractions, with ten more roundings for forming the inputs; F~'
    are the metric-folded fluxes minus the base state's (what the perturbation
    form contracts), dF the face terms.

    Input: the state enters as q' = q - q0 rounded to float32, so each face
    node's dissipation term lambda (q'+ - q'-) / 2 of the LLF flux may move by
    up to lambda u (|q'-| + |q'+|) / 2 even where the exact term vanishes
    (continuous fields: float64 traces that differ in their last bits round
    to the same float32); lifted with Fscale and |LIFT|. Per element the
    largest |q'| of the element and of the face's neighbour, and the largest
    |u| + c of the whole state, stand in for the node values.

    Computed in float64 from the oracle's parts; ``parts=True`` returns the
    arithmetic and the input term separately."""
    ref, g = osol.ref, osol.g
    Ft, dF = osol.rhs_parts(q)
    base = np.zeros_like(q)
    base[:, 0] = gas.rho0
    base[:, 4] = gas.p0 / (gas.gamma - 1.0)
    Ft0, _ = osol.rhs_parts(base)
    D = (ref.Dr, ref.Ds, ref.Dt)
    A = sum(np.einsum("ij,kvj->kvi", np.abs(D[a]), np.abs(Ft[:, a] - Ft0[:, a])) for a in range(3))
    A = A + np.einsum("ij,kvj->kvi", np.abs(ref.LIFT), np.abs(dF))
    K = 3 * ref.Np + 4 * ref.Nfp
    # input rounding of the LLF dissipation term
    rho = q[:, 0]
    u = q[:, 1:4] / rho[:, None]
    pr = (gas.gamma - 1.0) * (q[:, 4] - 0.5 * rho * np.sum(u * u, axis=1))
    lam = np.max(np.sqrt(np.sum(u * u, axis=1)) + np.sqrt(gas.gamma * np.abs(pr) / rho))
    qp = np.abs(q - base).max(axis=2)                                   # [K, 5]
    jump = 0.5 * lam * U32 * (qp[:, None, :] + qp[g.EToE])              # [K, 4, 5]
    dF_in = np.repeat((g.Fscale[:, :, None] * jump).transpose(0, 2, 1), ref.Nfp, axis=2)
    arith = (K + 10) * U32 * A
    inp = np.einsum("ij,kvj->kvi", np.abs(ref.LIFT), dF_in)
    return (arith, inp) if parts else arith + inp


U64 = 2.0 ** -53          # unit roundoff of float64


def f64_oracle_bound(osol, q, gas):
    """Rounding bound of the float64 oracle's own right-hand side, which works
    on the total state (base state included):
    (K + 10) u64 (sum_a |D_a| |F~_a| + |LIFT| |dF|) for the contractions, plus
    64 u64 |LIFT| Fscale M for the face terms, M = (|n.F-| + |n.F+|) / 2 +
    lambda (|q-| + |q+|) / 2 bounded by element maxima: traces, characteristic
    ghosts (square roots and powers) and fluxes carry a few tens of roundings
    of quantities of that size before they cancel. The float32 perturbation
    form does not see these roundings (at rest it computes exact zeros), so
    a comparison of the two must allow them."""
    ref, g = osol.ref, osol.g
    Ft, dF = osol.rhs_parts(q)
    D = (ref.Dr, ref.Ds, ref.Dt)
    A = sum(np.einsum("ij,kvj->kvi", np.abs(D[a]), np.abs(Ft[:, a])) for a in range(3))
    A = A + np.einsum("ij,kvj->kvi", np.abs(ref.LIFT), np.abs(dF))
    K = 3 * ref.Np + 4 * ref.Nfp
    rho = q[:, 0]
    u = q[:, 1:4] / rho[:, None]
    pr = (gas.gamma - 1.0) * (q[:, 4] - 0.5 * rho * np.sum(u * u, axis=1))
    lam = np.max(np.sqrt(np.sum(u * u, axis=1)) + np.sqrt(gas.gamma * np.abs(pr) / rho))
    fl = np.stack([q[:, 1:4],                                             # [K, 5, 3, Np]
                   q[:, 1:2] * u + pr[:, None] * np.eye(3)[0][:, None],
                   q[:, 2:3] * u + pr[:, None] * np.eye(3)[1][:, None],
                   q[:, 3:4] * u + pr[:, None] * np.eye(3)[2][:, None],
                   u * (q[:, 4] + pr)[:, None]], axis=1)
    fmax = np.abs(fl).max(axis=(2, 3))                                    # [K, 5]
    qabs = np.abs(q).max(axis=2)
    M = 0.5 * (fmax[:, None, :] + fmax[g.EToE]) + 0.5 * lam * (qabs[:, None, :] + qabs[g.EToE])
    dF_in = np.repeat((g.Fscale[:, :, None] * M).transpose(0, 2, 1), ref.Nfp, axis=2)
    return (K + 10) * U64 * A + 64 * U64 * np.einsum("ij,kvj->kvi", np.abs(ref.LIFT), dF_in)


def f32_parity_bound(osol, q, gas):
    """What a float32-form result may differ from the float64 oracle by:
    the float32 form's rounding plus the oracle's own."""
    return f32_contraction_bound(osol, q, gas) + f64_oracle_bound(osol, q, gas)


# Orientation convention of dg_upload_geometry (include/dg_euler.h): face
# vertex c of face f of element e is face vertex PERMS[o][c] of the
# neighbour's face.
FACE_VERTS = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))
PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def orientation_codes(EToV, EToE, EToF):
    K = len(EToV)
    ori = np.zeros((K, 4), dtype=np.int8)
    for e in range(K):
        for f in range(4):
            e2 = int(EToE[e, f])
            if e2 < 0:
                continue
            f2 = int(EToF[e, f])
            for o, P in enumerate(PERMS):
                if all(EToV[e][FACE_VERTS[f][c]] == EToV[e2][FACE_VERTS[f2][P[c]]] for c in range(3)):
                    ori[e, f] = o
                    break
            else:
                raise ValueError("faces do not match")
    return ori


def inflow_case(p, seed=13):
    """Kuhn cube with the faces on x = -1 tagged 1 (the inflow pulse of
    section 2.4) and every other boundary face tagged 0."""
    from oracle.geometry import Geometry
    from oracle.reference_element import ReferenceElement
    from paper_1710_03887_gb300 import workloads as W
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=seed)
    geom = Geometry(ReferenceElement(p), xyz, EToV)
    fx = geom.x[:, geom.ref.Fmask].mean(axis=2)[..., 0]          # face centroids' x, [K, 4]
    tag = np.where(geom.boundary, np.where(fx < -1.0 + 1e-9, 1, 0), -1).astype(np.int8)
    return xyz, EToV, geom, tag
