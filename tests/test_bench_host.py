"""Host-side pieces of bench.py (no GPU): the clock record's parsing of
nvidia-smi's CSV, the ncu-summary lookup that withholds traffic once a
kernel's source has changed, and the algorithmic counts behind the
roofline at the p = 3 workload."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _line(sm, smax, hw="Not Active", thermal="Not Active", sw_thermal="Not Active", power="Not Active"):
    return f"0, {sm}, {smax}, 900.00, 0x0000000000000000, {hw}, {thermal}, {sw_thermal}, {power}"


def test_clock_record_median_and_reasons(bench):
    c = bench.ClockSampler(-1)
    c.lines = [_line(1000, 2070), _line(1965, 2070), _line(1980, 2070, power="Active"),
               _line(1995, 2070), _line(1950, 2070, hw="Active")]
    c.skip = 1                                   # the first sample came before the region
    out = c.summary()
    assert out["samples"] == 4
    assert out["sm_mhz"] == pytest.approx(1972.5)
    assert out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_record_of_a_short_region_and_of_none(bench):
    c = bench.ClockSampler(-1)
    c.lines = [_line(1900, 2070)]
    c.skip = 1
    out = c.summary()
    assert out["sm_mhz"] == 1900 and "note" in out
    c.lines, c.skip = [], 0
    assert c.summary()["reasons"] == ["unsampled"]


def test_traffic_is_withheld_when_the_kernel_changed(bench, tmp_path, monkeypatch):
    import hashlib
    src = open(os.path.join(ROOT, "paper_1710_03887_gb300", "csrc", "stage_f32.cu"), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    prof = tmp_path / "profiles"
    csrc = tmp_path / "paper_1710_03887_gb300" / "csrc"
    prof.mkdir()
    csrc.mkdir(parents=True)
    (csrc / "stage_f32.cu").write_bytes(src)
    (prof / "k.md").write_text(f"source_sha256_16: {sha}\nbytes_per_launch_full: 123456\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k.md", "stage_f32.cu") == 123456.0
    (csrc / "stage_f32.cu").write_bytes(src + b"\n// changed\n")
    assert bench.profiled_traffic("k.md", "stage_f32.cu") is None
    assert bench.profiled_traffic("missing.md", "stage_f32.cu") is None


def test_algorithmic_counts_at_p3(bench):
    # 20 nodes, 10 face nodes: (103 + 25) per node, 30 Np^2, 101 per face
    # node, 40 Np Nfp (1 FMA = 2 flops)
    assert bench.stage_flops_per_element(3) == 20 * 128 + 30 * 400 + 40 * 101 + 40 * 200
    # q and res read and written (4 x 5 x Np words), 32 words of geometry, 16 B of connections
    assert bench.stage_bytes_per_element(3, 4) == 4 * 5 * 20 * 4 + 32 * 4 + 16 == 1744
    assert bench.stage_bytes_per_element(3, 8) == 3472


def test_repeat_stats_median_and_spread(bench):
    out = bench.repeat_stats([23.0, 22.0, 25.0, 22.5, 24.0], 20, sm_mhz=2000.0)
    assert out["n"] == 5
    assert out["median_ms_per_step"] == pytest.approx(23.0 / 20)
    assert out["min_ms_per_step"] == pytest.approx(22.0 / 20)
    assert out["max_ms_per_step"] == pytest.approx(25.0 / 20)
    assert out["spread_rel"] == pytest.approx(3.0 / 23.0)
    assert out["median_ms_per_step_x_sm_mhz"] == pytest.approx(23.0 / 20 * 2000.0)


def test_acoustic_energy_of_a_uniform_field(bench):
    """On one element of the reference tetrahedron mapped with Jacobian J, a
    uniform p' and m' give (p'^2/(2 rho0 c0^2) + |m'|^2/(2 rho0)) times the
    volume 4/3 J (the mass matrix sums to the reference volume)."""
    import numpy as np
    from oracle.reference_element import ReferenceElement
    ref = ReferenceElement(2)
    gamma, rho0, p0 = 1.4, 1.225, 101325.0
    q = np.zeros((1, 5, ref.Np))
    q[0, 4] = 50.0          # p'
    q[0, 1] = 0.3
    q[0, 3] = -0.4          # |m'| = 0.5
    J = np.array([0.7])
    c2 = gamma * p0 / rho0
    want = (50.0 ** 2 / (2 * rho0 * c2) + 0.25 / (2 * rho0)) * 4.0 / 3.0 * 0.7
    assert bench.acoustic_energy(q, J, ref.M, gamma, rho0, p0) == pytest.approx(want, rel=1e-13)


def test_precision_comparison_figures(bench):
    """Known differences between two synthetic runs come out as the stated
    relative figures; identical runs give zeros."""
    import numpy as np
    from oracle.reference_element import ReferenceElement
    ref = ReferenceElement(1)
    gamma, rho0, p0 = 1.4, 1.225, 101325.0
    E0 = p0 / (gamma - 1.0)
    K, Np = 3, ref.Np
    rng = np.random.default_rng(0)
    q0 = np.zeros((K, 5, Np))
    q0[:, 0] = rho0
    q0[:, 4] = E0 * (1.0 + 0.1 * rng.random((K, Np)))        # a pressure pulse at rest
    q64 = q0.copy()
    q64[:, 1] = 2.0 * rng.standard_normal((K, Np))
    q64[:, 4] += 0.01 * E0
    probes64 = np.repeat(q64[:1, :, :1].transpose(0, 2, 1), 6, axis=1).repeat(4, axis=0)  # [4, 6, 5]
    tot0 = np.array([5.0, 0.0, 0.0, 0.0, 1e6])
    run64 = dict(q0=q0, q=q64, probes=probes64, tot0=tot0, tot=tot0 + 1e-3, led=np.full(5, -1e-3),
                 J=np.ones(K))
    same = bench.precision_comparison(dict(run64), run64, 0.1, ref.M, gamma, rho0, p0)
    assert max(same["max_err_per_var_rel_to_perturbation"]) == 0.0
    assert same["pressure_max_diff_rel_to_pulse_amplitude"] == 0.0
    assert same["energy_of_difference_rel_to_initial_acoustic_energy"] == 0.0
    assert same["axis_probes_f32_minus_fp64_max_rel_to_pulse_amplitude"] == 0.0
    assert max(same["balance_rel_fp64"]) < 1e-15
    q32 = q64.copy()
    q32[1, 4, 0] += 3.0 * E0 * 1e-6            # energy (= pressure / (gamma - 1)) only
    probes32 = probes64.copy()
    probes32[2, 5, 4] += 7.0                    # step 2, probe 5, energy
    run32 = dict(run64, q=q32, probes=probes32, led=run64["led"] + 2e-3)
    out = bench.precision_comparison(run32, run64, 0.1, ref.M, gamma, rho0, p0)
    err = out["max_err_per_var_rel_to_perturbation"]
    assert err[:4] == [0.0, 0.0, 0.0, 0.0]
    assert err[4] == pytest.approx(3.0 * E0 * 1e-6 / np.abs(q64[:, 4] - E0).max())
    assert out["pressure_max_diff_rel_to_pulse_amplitude"] == pytest.approx(
        (gamma - 1.0) * 3.0 * E0 * 1e-6 / (0.1 * p0))
    assert out["axis_probes_f32_minus_fp64_max_rel_to_pulse_amplitude"] == pytest.approx(
        (gamma - 1.0) * 7.0 / (0.1 * p0))
    assert out["axis_probes_spread_rel_to_pulse_amplitude"]["f32"] == pytest.approx(
        (gamma - 1.0) * 7.0 / (0.1 * p0))
    assert out["axis_probes_spread_rel_to_pulse_amplitude"]["fp64"] == 0.0
    assert out["balance_rel_f32"][0] == pytest.approx(2e-3 / 5.0)
    c0 = np.sqrt(gamma * p0 / rho0)
    assert out["balance_rel_f32"][2] == pytest.approx(2e-3 / (5.0 * c0))   # momentum: mass x c0
    assert out["ledger_f32_minus_fp64_rel_to_totals"][4] == pytest.approx(2e-3 / 1e6)


def test_far_field_probes_cover_the_front_half_sphere(bench):
    import numpy as np
    p = bench.far_field_probes(32, 2.5)
    assert p.shape == (32, 3)
    np.testing.assert_allclose(np.linalg.norm(p, axis=1), 2.5, rtol=1e-14)
    assert np.all(p[:, 0] > 0)
    # spread: no two probes closer than a fifth of the mean spacing on the half-sphere
    d = np.linalg.norm(p[:, None] - p[None], axis=2) + np.eye(32) * 1e9
    assert d.min() > 0.2 * np.sqrt(2 * np.pi * 2.5 ** 2 / 32)
