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
