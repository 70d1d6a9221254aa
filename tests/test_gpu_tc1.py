"""The one-pass tensor-core variant (DG_PREC_F32_TC1) against the float64
oracle (GPU).

The variant gives the float32 operands of both contractions (volume and
LIFT, Eq. 10) to the tensor cores as they are: kind::tf32 reads them as
tf32, keeping 10 of float32's 23 mantissa bits, so each operand carries a
relative error below u_t = 2^-10 (truncation) and each product below
2 u_t + u_t^2. The bound at every node and variable is therefore

    (2 u_t + u_t^2) (sum_a |D_a| |F~'_a| + |LIFT| |dF|)  +  the float32 bound

(the float32 bound: accumulation over K terms, input rounding;
tests/_cases.py f32_contraction_bound). The same bound with u_t = 2^-11
(round to nearest) would fail where the hardware truncates; the test reports
the largest ratio to the bound. The float32 forms stay at float32 level
(tests/test_gpu_f32.py); this variant is measured, in the bench's `forms`,
with its error against float64.
"""
import numpy as np
import pytest

from paper_1710_03887_gb300 import workloads as W

from ._cases import CHARACTERISTIC, FREESTREAM, SLIP_WALL, Case, direction_tags, f32_contraction_bound

pytestmark = pytest.mark.gpu

UT = 2.0 ** -10            # tf32 operand: 10 stored mantissa bits, truncated


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_one_pass_rhs_within_the_tf32_bound(cuda_device, p):
    from paper_1710_03887_gb300 import binding as B
    xyz, EToV = W.kuhn_cube(3, jitter=0.12, seed=p)
    probe = Case(p, xyz, EToV)
    tags = direction_tags(xyz, EToV, probe.geom)
    case = Case(p, xyz, EToV, tags=tags, modes={0: CHARACTERISTIC, 1: FREESTREAM, 2: SLIP_WALL})
    q = case.smooth(0.05, seed=p)
    ref = case.oracle.rhs(q)
    arith, inp = f32_contraction_bound(case.oracle, q, case.gas, parts=True)
    K = 3 * case.ref.Np + 4 * case.ref.Nfp
    A = arith / ((K + 10) * 2.0 ** -24)                  # sum_a |D_a||F~'_a| + |LIFT||dF|
    bound = (2 * UT + UT * UT) * A + arith + inp
    S = B.Solver(p, precision=B.DG_PREC_F32_TC1, **case.gas_kw)
    S.upload_mesh(case.xyz, case.EToV, face_tag=case.tags)
    for ident, mode in case.modes.items():
        S.set_bc(ident, mode)
    S.set_state(q)
    got = S.eval_rhs()
    ratio = np.abs(got - ref) / bound
    print(f"p={p}: max |error| / bound = {ratio.max():.3f}")
    assert np.all(np.isfinite(got))
    assert ratio.max() <= 1.0
    # and the variant really is less accurate than the float32 forms: its
    # error exceeds the float32 bound somewhere (the operands are tf32)
    assert np.any(np.abs(got - ref) > arith + inp)


def test_one_pass_run_is_finite_and_close_to_the_float32_form(cuda_device):
    """20 steps of the C1 pulse: the one-pass variant stays finite and
    within 1e-2 of the perturbation of the float32 form's run (the
    right-hand side's ~1e-3 relative error, integrated)."""
    from paper_1710_03887_gb300 import binding as B
    xyz, EToV = W.kuhn_cube(6)
    out = {}
    for prec in (B.DG_PREC_F32, B.DG_PREC_F32_TC1):
        S = B.Solver(1, precision=prec, gamma=W.GAMMA, rho0=W.RHO0_SI, p0=W.P0_SI)
        S.upload_mesh(xyz, EToV)
        q0 = W.gaussian_pulse_state(S.node_coords(), W.GAMMA, W.RHO0_SI, W.P0_SI, 0.005, 0.15)
        dt = S.stable_dt(q0, 0.5)
        S.set_state(q0)
        S.step(20, dt)
        out[prec], _ = S.get_state()
        S.close()
    base = W.uniform_state(q0.shape[0], q0.shape[2], W.RHO0_SI, (0, 0, 0), W.P0_SI, W.GAMMA)
    a, b = out[B.DG_PREC_F32_TC1], out[B.DG_PREC_F32]
    assert np.all(np.isfinite(a))
    num = np.abs(a - b).max(axis=(0, 2))
    den = np.abs(b - base).max(axis=(0, 2))
    assert np.all(num[[0, 4]] <= 1e-2 * den[[0, 4]]), num / den
    assert np.all(num[1:4] <= 1e-2 * den[1:4].max()), num / den
