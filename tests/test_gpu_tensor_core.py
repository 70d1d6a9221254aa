"""Unit probe of the tcgen05 building blocks (tc_ptx.cuh) on the GPU.

One CTA multiplies a 128 x K by a K x N operand (tf32 in, float32 out)
through the same descriptor layout the stage kernel uses; the product is
checked against float64 host arithmetic on the same tf32-rounded inputs.
"""
import ctypes
import subprocess
from pathlib import Path

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parent.parent
SRC = ROOT / "tests" / "cuda" / "tc_gemm_probe.cu"
OUT = ROOT / "paper_1710_03887_gb300" / "_build" / "tc_gemm_probe.so"


def tf32_round(x):
    """Round float32 to tf32 (10 explicit mantissa bits), nearest, ties away from zero."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def probe():
    from paper_1710_03887_gb300 import build_lib
    OUT.parent.mkdir(exist_ok=True)
    if not OUT.exists() or OUT.stat().st_mtime < SRC.stat().st_mtime:
        subprocess.run([build_lib._nvcc(), *build_lib.ARCH, "-O2", "-std=c++17", "-Xcompiler",
                        "-fPIC", "-shared", "-o", str(OUT), str(SRC)], check=True)
    lib = ctypes.CDLL(str(OUT))
    lib.tc_gemm_probe.restype = ctypes.c_int
    lib.tc_gemm_probe.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("N,K", [(16, 8), (32, 104), (16, 56), (32, 24)])
def test_tf32_mma_matches_host(cuda_device, probe, N, K):
    import torch
    rng = np.random.default_rng(N * 1000 + K)
    A = rng.normal(size=(128, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32)
    dA = torch.from_numpy(A).to(cuda_device)
    dB = torch.from_numpy(B).to(cuda_device)
    dD = torch.full((128, N), float("nan"), dtype=torch.float32, device=cuda_device)
    st = torch.zeros(1, dtype=torch.int32, device=cuda_device)
    rc = probe.tc_gemm_probe(dA.data_ptr(), dB.data_ptr(), dD.data_ptr(), N, K, st.data_ptr())
    assert rc == 0
    assert int(st.item()) == 0, "MMA completion wait timed out"
    ref = tf32_round(A).astype(np.float64) @ tf32_round(B).astype(np.float64).T
    got = dD.cpu().numpy()
    scale = np.abs(tf32_round(A)).astype(np.float64) @ np.abs(tf32_round(B)).astype(np.float64).T
    assert np.all(np.abs(got - ref) <= 1e-6 * scale + 1e-30), np.abs(got - ref).max()


def test_tf32_mma_m64_rows_in_tensor_memory(cuda_device, probe):
    """M = 64: the same product, with every lane of the accumulator read back;
    each of the 64 result rows must appear, whole and correct, in exactly one
    tensor-memory lane (the stage kernel's M = 64 tiles rely on the mapping
    this test prints and pins)."""
    import torch
    probe.tc_gemm_probe_m64.restype = ctypes.c_int
    probe.tc_gemm_probe_m64.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int,
                                                               ctypes.c_void_p]
    N, K = 24, 104
    rng = np.random.default_rng(64)
    A = rng.normal(size=(64, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32)
    dA = torch.from_numpy(A).to(cuda_device)
    dB = torch.from_numpy(B).to(cuda_device)
    dD = torch.full((128, 32), float("nan"), dtype=torch.float32, device=cuda_device)
    st = torch.zeros(1, dtype=torch.int32, device=cuda_device)
    rc = probe.tc_gemm_probe_m64(dA.data_ptr(), dB.data_ptr(), dD.data_ptr(), N, K, st.data_ptr())
    assert rc == 0
    assert int(st.item()) == 0, "MMA completion wait timed out"
    ref = tf32_round(A).astype(np.float64) @ tf32_round(B).astype(np.float64).T
    scale = np.abs(tf32_round(A)).astype(np.float64) @ np.abs(tf32_round(B)).astype(np.float64).T
    got = dD.cpu().numpy()[:, :N].astype(np.float64)
    lanes = []
    for r in range(64):
        hit = [L for L in range(128)
               if np.all(np.abs(got[L] - ref[r]) <= 1e-6 * scale[r] + 1e-30)]
        lanes.append(hit)
    print("M=64 row -> tensor-memory lanes:", [h[0] if len(h) == 1 else h for h in lanes])
    assert all(len(h) == 1 for h in lanes)
    # row r sits in lane 32 (r // 16) + r % 16: the first 16 lanes of each
    # warp's quarter of tensor memory
    assert [h[0] for h in lanes] == [32 * (r // 16) + r % 16 for r in range(64)]


def test_network_tanh_against_tanhf(cuda_device, probe):
    """The closure network's tanh (1 - 2 / (1 + e^{2x}) with hardware exp2 and
    reciprocal) stays within 3e-7 of CUDA's tanhf everywhere, including the
    saturated tails and x = 0."""
    import torch
    probe.tanh_probe.restype = ctypes.c_int
    probe.tanh_probe.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    x = np.concatenate([np.linspace(-30.0, 30.0, 200001), [0.0, -0.0, 1e-30, -1e-30, 1e-6, 88.0, -88.0,
                                                           1e30, -1e30]]).astype(np.float32)
    dx = torch.from_numpy(x).to(cuda_device)
    fast = torch.empty_like(dx)
    ref = torch.empty_like(dx)
    assert probe.tanh_probe(dx.data_ptr(), fast.data_ptr(), ref.data_ptr(), x.size) == 0
    f, r = fast.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(f))
    assert np.abs(f - r).max() <= 3e-7, np.abs(f - r).max()
    assert np.abs(f - np.tanh(x.astype(np.float64))).max() <= 3e-7


def test_bounded_completion_wait_gives_up_and_the_device_stays_usable(cuda_device, probe):
    """The stage kernel's tensor-core completion wait is bounded: here nothing
    ever arrives at the barrier, so the wait gives up after its tries, sets
    the status word and frees its tensor memory; the same process then runs
    a normal product."""
    import time
    import torch
    probe.tc_wait_timeout_probe.restype = ctypes.c_int
    probe.tc_wait_timeout_probe.argtypes = [ctypes.c_uint, ctypes.c_void_p]
    st = torch.zeros(3, dtype=torch.int32, device=cuda_device)
    t0 = time.perf_counter()
    assert probe.tc_wait_timeout_probe(1 << 12, st.data_ptr()) == 0
    assert time.perf_counter() - t0 < 10.0
    status, cleanup_tries, other_parity_tries = (int(v) for v in st.cpu())
    assert status == 1
    # the cleanup wait (on the parity that timed out) really waits, to its
    # limit; the flipped parity would have returned at the first try
    assert cleanup_tries == 1 << 12
    assert other_parity_tries == 0
    test_tf32_mma_matches_host(cuda_device, probe, 16, 8)


def test_float64_newton_reciprocal_and_sqrt(cuda_device, probe):
    """The float64 stage's reciprocal and square root (Newton-Raphson from
    the hardware estimates) stay within 2 ulp of the correctly rounded
    division and sqrt over the range a state can reach."""
    import torch
    probe.fp64_nr_probe.restype = ctypes.c_int
    probe.fp64_nr_probe.argtypes = [ctypes.c_void_p] * 5 + [ctypes.c_int]
    rng = np.random.default_rng(5)
    x = np.concatenate([10.0 ** rng.uniform(-8, 12, size=200000),
                        [1.0, 2.0, 0.5, 1.225, 101325.0, 1.4, 3.0, 1e-300, 1e300]])
    dx = torch.from_numpy(x).to(cuda_device)
    outs = [torch.empty_like(dx) for _ in range(4)]
    assert probe.fp64_nr_probe(dx.data_ptr(), *(o.data_ptr() for o in outs), x.size) == 0
    rcp, rcp_ref, sq, sq_ref = (o.cpu().numpy() for o in outs)
    ok = (x > 1e-290) & (x < 1e290)
    ulp = np.spacing(np.abs(rcp_ref))
    assert np.all(np.abs(rcp - rcp_ref)[ok] <= 2 * ulp[ok])
    ulp = np.spacing(sq_ref)
    assert np.all(np.abs(sq - sq_ref)[ok] <= 2 * ulp[ok])
