"""The debug build's device bounds checks (GPU).

`compute-sanitizer` is not available on this machine, so the library has a
debug variant, libdgeuler_debug.so: the same sources compiled with
-DDG_BOUNDS_CHECK, in which every index a kernel reads from the mesh tables
(face lists, connection words, node and face-node tables, boundary slots,
halo rows) is checked before the access it selects; a failed check skips
the access and latches a status bit that the host reports as DG_ERR_BOUNDS.

* Every case of tests/_bounds_cases.py (all forms, all face orientations,
  a short last tile, every boundary kind, probes, the learned closure, two
  emulated partition ranks) runs on the debug build with no check failing,
  and gives the release build's results: the checks change no arithmetic,
  so every state, probe series and ledger is bitwise equal.
* A check made to fail on purpose (no out-of-range access: a condition
  nothing meets) reaches the host as DG_ERR_BOUNDS and is cleared; the
  context goes on cleanly.
* The release build reports no checks and refuses the self-test.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import build_lib

from . import _bounds_cases as BC

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_runs_every_case_clean_and_bitwise_equal(cuda_device, tmp_path):
    build_lib.build(debug=True)
    rel = BC.run_all()
    out = tmp_path / "debug.npz"
    env = dict(os.environ, DG_EULER_BUILD="debug")
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); "
            f"from tests._bounds_cases import main; main({str(out)!r})")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    dbg = np.load(out)
    assert int(dbg["flags"]) == B.DG_BUILD_BOUNDS_CHECKS
    # the failed check on purpose: reported once, then a clean step
    assert dbg["selftest"].tolist() == [B.DG_ERR_BOUNDS, 0]
    for k, v in rel.items():
        assert np.isfinite(v).all(), k
        np.testing.assert_array_equal(dbg[k], v, err_msg=k)


def test_release_build_has_no_checks(cuda_device):
    assert B.build_flags() == 0
    xyz, E, tags = BC.mesh()
    S = B.Solver(2, **BC.SI)
    S.upload_mesh(xyz, E, face_tag=tags)
    with pytest.raises(B.DGError) as e:
        S.bounds_selftest()
    assert e.value.code == B.DG_ERR_UNSUPPORTED
    S.close()
