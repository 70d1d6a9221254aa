"""dg_weighted_totals_static: conserved totals for callers that cannot allocate.

Callers whose device memory belongs to another allocator, or that sit inside
a running time loop where cudaMalloc/cudaFree must not be called, get the
totals from this entry point: it takes only their own device buffers and
keeps its partial sums in a static device array of the library. The test
checks it against dg_conserved_totals (the allocating path of the same
reduction) on two calls in a row, through the C ABI.
"""
import ctypes

import numpy as np
import pytest

from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-13   # same float64 sums, different block decomposition


def _totals_static(lib, q, J, w, K, Np, out, stream):
    return lib.dg_weighted_totals_static(q.data_ptr(), J.data_ptr(), w.data_ptr(), K, Np,
                                         out.data_ptr(), stream)


def test_static_totals_match_allocating_totals(cuda_device):
    import torch
    lib = B.load()
    p = 1
    xyz, EToV = W.kuhn_cube(12)                       # 10,368 elements: three partial blocks
    S = B.Solver(p, W.GAMMA, W.RHO0_SI, W.P0_SI)
    stream = torch.cuda.current_stream(cuda_device)
    S.set_stream(stream.cuda_stream)
    S.upload_mesh(xyz, EToV)
    q0 = W.gaussian_pulse_state(S.node_coords(), W.GAMMA, W.RHO0_SI, W.P0_SI, 0.2, 0.5,
                                center=(0.3, -0.2, 0.1))
    q0[:, 1] += 3.0                                   # nonzero momentum totals
    S.set_state(q0)
    K, Np = S.K, S.Np
    J = torch.from_numpy(S.geometry()["J"]).to(cuda_device)
    w = torch.from_numpy(ReferenceElement(p).M.sum(axis=0)).to(cuda_device)
    q = torch.empty((K, 5, Np), dtype=torch.float64, device=cuda_device)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device=cuda_device)
    dt = S.stable_dt(q0)
    for call in range(2):                             # two calls in a row, different states
        if call == 1:
            S.step(3, dt)
        S.get_state(q)
        ref = S.totals()
        rc = _totals_static(lib, q, J, w, K, Np, out, stream.cuda_stream)
        assert rc == B.DG_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=RTOL, atol=RTOL * np.abs(ref).max())
    # sizes beyond the stated maximum are rejected before any memory is touched
    too_many = int(lib_max_elements())
    assert _totals_static(lib, q, J, w, too_many + 1, Np, out, stream.cuda_stream) == B.DG_ERR_ARG
    assert _totals_static(lib, q, J, w, K, 36, out, stream.cuda_stream) == B.DG_ERR_ARG
    assert lib.dg_weighted_totals_static(None, J.data_ptr(), w.data_ptr(), K, Np,
                                         out.data_ptr(), stream.cuda_stream) == B.DG_ERR_ARG


def lib_max_elements():
    import re
    from pathlib import Path
    text = (Path(__file__).resolve().parent.parent / "include" / "dg_euler.h").read_text()
    a, b = re.search(r"DG_STATIC_TOTALS_MAX_ELEMENTS \((\d+)LL \* (\d+)LL\)", text).groups()
    return int(a) * int(b)
