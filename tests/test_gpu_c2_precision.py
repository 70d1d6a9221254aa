"""The float32 perturbation form against plain float64 DG over the full 2000
steps of the ball configuration (a 10 % p0 pulse at the centre of a ball of
radius 1, p = 3, characteristic pass-through condition on the sphere), at a
reduced mesh size: the n = 10 lattice ball (6,000 tetrahedra, no jitter, so
the mesh has the symmetries of the cube). The time step is CFL 0.5 of that
mesh, so in 2000 steps the pulse travels ~0.9 of the radius and its front
crosses the sphere: the comparison covers the outgoing wave at the
pass-through boundary.

Both forms run through the C ABI on the GPU (bench.py's precision_run, the
code the bench's full-size section uses). The bounds, per result:

* state, per conserved variable, max |f32 - fp64| / max |fp64 - q0|: the
  float32 right-hand side is accurate to ~2e-5 of its largest value (its
  parity bound against the oracle), and a run accumulates that over 10,000
  stages with partial cancellation; bound 2e-3;
* pressure, max |p32 - p64| / (A p0): the scope's bar of 1e-3 of the pulse
  amplitude;
* energy of the difference field / initial acoustic energy: below (1e-3)^2;
* the six axis probes (images of one point under the mesh's symmetries):
  float32 against float64 within 1e-3 of the pulse amplitude; each form's
  spread across the six is its rounding (float64: 1e-9 of the amplitude,
  float32: 1e-3);
* conservation: totals(t) - totals(0) + ledger, relative to the totals, at
  float64 rounding for the float64 form (1e-12) and at the float32 rounding
  of the stored perturbation for the float32 form (1e-7); the two ledgers
  agree to 1e-6 of the totals.
"""
import importlib.util
import os

import numpy as np
import pytest

from paper_1710_03887_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 2000
AMPLITUDE, WIDTH = 0.1, 0.15


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def fp64_run(cuda_device, bench):
    import torch
    from paper_1710_03887_gb300 import binding as B
    xyz, EToV = W.ball(10, 1.0)
    stream = torch.cuda.current_stream(cuda_device)
    return bench.precision_run(3, xyz, EToV, B.DG_PREC_FP64, STEPS, AMPLITUDE, WIDTH, 0.5,
                               cuda_device, stream)


@pytest.mark.parametrize("form", ["f32", "f32_tc"])
def test_f32_against_fp64_over_2000_steps(cuda_device, bench, fp64_run, form):
    """Both float32 forms (SIMT and tensor-core contractions) against the
    float64 run, with the same bars."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    xyz, EToV = W.ball(10, 1.0)
    stream = torch.cuda.current_stream(cuda_device)
    # bench.AXIS_PROBES: images of one point inside an element under the
    # mesh's reflections and axis swaps (the lattice symmetries), so the
    # discrete solution of a centred pulse is equal at all six
    r64 = fp64_run
    prec = {"f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC}[form]
    r32 = bench.precision_run(3, xyz, EToV, prec, STEPS, AMPLITUDE, WIDTH, 0.5, cuda_device,
                              stream)
    c0 = np.sqrt(W.GAMMA * W.P0_SI / W.RHO0_SI)
    assert c0 * r64["dt"] * STEPS > 0.8          # the front has reached the sphere
    out = bench.precision_comparison(r32, r64, AMPLITUDE, B.reference_mass(3), W.GAMMA,
                                     W.RHO0_SI, W.P0_SI)
    print(out)
    assert np.all(np.array(out["max_err_per_var_rel_to_perturbation"]) < 2e-3), out
    assert out["pressure_max_diff_rel_to_pulse_amplitude"] < 1e-3, out
    assert out["energy_of_difference_rel_to_initial_acoustic_energy"] < 1e-6, out
    assert out["axis_probes_f32_minus_fp64_max_rel_to_pulse_amplitude"] < 1e-3, out
    assert out["axis_probes_spread_rel_to_pulse_amplitude"]["fp64"] < 1e-9, out
    assert out["axis_probes_spread_rel_to_pulse_amplitude"]["f32"] < 1e-3, out
    # the probes saw the pulse pass (not a trivially quiet comparison)
    assert out["axis_probes_peak_rel_to_pulse_amplitude"] > 0.05, out
    assert np.all(np.array(out["balance_rel_fp64"]) < 1e-12), out
    assert np.all(np.array(out["balance_rel_f32"]) < 1e-7), out
    assert np.all(np.array(out["ledger_f32_minus_fp64_rel_to_totals"]) < 1e-6), out
