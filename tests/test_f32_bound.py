"""The float32 rounding bound the GPU parity tests hold the float32 forms to
(tests/_cases.f32_contraction_bound), checked on the CPU against float32
emulations of the two things it bounds:

* the contractions: Eq. 10's volume and LIFT products formed from the
  float64 parts rounded to float32 and multiplied in float32 (numpy's
  float32 product), against the float64 products;
* the input rounding: the oracle's right-hand side at q0 + fl32(q - q0)
  against the one at q, on a mesh and state where the exact face jumps
  vanish (continuous pulse at rest), so the bound's input term is all that
  covers the difference."""
import numpy as np

from oracle.euler_dg import CHARACTERISTIC, INFLOW_PULSE, SLIP_WALL, Gas
from oracle.euler_dg import Solver as OSolver
from oracle.geometry import Geometry
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import workloads as W

from ._cases import SI, f32_contraction_bound, f64_oracle_bound

GAS = Gas(SI["gamma"], SI["rho0"], SI["p0"])


def _base(q):
    b = np.zeros_like(q)
    b[:, 0] = GAS.rho0
    b[:, 4] = GAS.p0 / (GAS.gamma - 1.0)
    return b


def test_bound_covers_float32_contractions():
    xyz, EToV = W.kuhn_cube(3, jitter=0.12, seed=4)
    g = Geometry(ReferenceElement(3), xyz, EToV)
    orc = OSolver(g, GAS)
    q = W.random_smooth_state(g.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, seed=3)
    Ft, dF = orc.rhs_parts(q)
    Ft0, _ = orc.rhs_parts(_base(q))
    ref = orc.ref
    D = (ref.Dr, ref.Ds, ref.Dt)
    exact = -sum(np.einsum("ij,kvj->kvi", D[a], Ft[:, a] - Ft0[:, a]) for a in range(3)) \
        + np.einsum("ij,kvj->kvi", ref.LIFT, dF)
    f = np.float32
    X = np.concatenate([(Ft[:, a] - Ft0[:, a]).astype(f) for a in range(3)] + [dF.astype(f)], axis=2)
    OT = np.concatenate([-D[a].T for a in range(3)] + [ref.LIFT.T], axis=0).astype(f)
    emul = (X.reshape(-1, X.shape[2]) @ OT).reshape(exact.shape).astype(np.float64)
    bound = f32_contraction_bound(orc, q, GAS)
    err = np.abs(emul - exact)
    assert np.all(err <= bound)
    assert err.max() > 0                      # the emulation does round


def test_bound_covers_input_rounding_where_jumps_vanish():
    xyz, EToV, tag, _ = W.horn_in_room(m1=1, room_length=0.03, room_half=0.03, growth=1.8,
                                       horn_length=0.1, aspect=3.0)
    g = Geometry(ReferenceElement(3), xyz, EToV)
    orc = OSolver(g, GAS, bc_id=np.where(tag < 0, 0, tag).astype(np.int64),
                  bc_mode={W.HORN_OUTER: CHARACTERISTIC, W.HORN_WALL: SLIP_WALL,
                           W.HORN_MOUTHPIECE: INFLOW_PULSE})
    q = W.gaussian_pulse_state(g.x, SI["gamma"], SI["rho0"], SI["p0"], 0.05, 0.01,
                               center=(0.1, 0.002, 0.0))
    base = _base(q)
    q32 = base + (q - base).astype(np.float32).astype(np.float64)
    diff = np.abs(orc.rhs(q32) - orc.rhs(q))
    arith, inp = f32_contraction_bound(orc, q, GAS, parts=True)
    assert np.all(diff <= arith + inp)
    # the arithmetic term alone does not cover the density here
    assert np.any(diff[:, 0] > arith[:, 0])


def test_oracle_bound_covers_its_rounding_at_rest():
    """At rest the exact right-hand side is zero with every boundary kind
    (walls, characteristic, the inflow at t = 0): what the oracle returns is
    its own rounding, which its bound must cover, on a fine graded mesh
    whose small elements make the terms large."""
    xyz, EToV, tag, _ = W.horn_in_room(m1=2, room_length=0.05, room_half=0.06, growth=1.5,
                                       horn_length=0.1, aspect=1.0)
    g = Geometry(ReferenceElement(3), xyz, EToV)
    orc = OSolver(g, GAS, bc_id=np.where(tag < 0, 0, tag).astype(np.int64),
                  bc_mode={W.HORN_OUTER: CHARACTERISTIC, W.HORN_WALL: SLIP_WALL,
                           W.HORN_MOUTHPIECE: INFLOW_PULSE})
    q = W.uniform_state(g.K, orc.ref.Np, SI["rho0"], (0, 0, 0), SI["p0"], SI["gamma"])
    r = np.abs(orc.rhs(q, 0.0))
    b = f64_oracle_bound(orc, q, GAS)
    assert np.all(r <= b)
    assert r[:, 4].max() > 0                  # there is rounding to cover
    # and the bound is not vacuous: within a few orders of the rounding seen
    assert b[:, 4].max() < 1e4 * r[:, 4].max()
