"""The boundary is a plain C interface (no GPU needed): the header compiles
as strict C99, and a C program linked against the in-tree library drives
the host-only entry points and the error paths through it, with no Python
in between."""
import shutil
import subprocess
from pathlib import Path

import pytest

from paper_1710_03887_gb300 import binding as B

ROOT = Path(__file__).resolve().parent.parent

PROGRAM = r"""
#include <stdio.h>
#include "dg_euler.h"

int main(void) {
  double rst[3 * 20];
  int32_t fmask[4 * 10];
  if (dg_reference_operators(3, rst, NULL, NULL, NULL, NULL, fmask) != DG_OK) return 1;
  int32_t nq = 0, nfq = 0;
  if (dg_modal_quadrature(2, NULL, NULL, &nq, &nfq) != DG_OK) return 2;
  dg_params prm = {1.4, 1.225, 101325.0, {0.0, 0.0, 0.0}, DG_BC_CHARACTERISTIC, DG_PREC_FP64};
  dg_ctx* ctx = NULL;
  if (dg_create(7, &prm, &ctx) != DG_ERR_UNSUPPORTED) return 3;
  if (dg_create(2, &prm, &ctx) != DG_OK) return 4;
  double xyz[] = {0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1};
  int32_t EToV[] = {0, 1, 2, 3};
  if (dg_upload_mesh(ctx, 4, xyz, 1, EToV, NULL, NULL) != DG_OK) return 5;
  int64_t K;
  int32_t Np, Nfp;
  if (dg_sizes(ctx, &K, &Np, &Nfp) != DG_OK || K != 1 || Np != 10 || Nfp != 6) return 6;
  int64_t pair[4 * 6];
  if (dg_face_pairs(ctx, pair, NULL) != DG_OK) return 7;
  for (int i = 0; i < 24; ++i)
    if (pair[i] != -1) return 8;
  if (dg_step(ctx, 1, 1e-3) != DG_ERR_ORDER) return 9;
  printf("%d %d %.17g %d\n", nq, nfq, rst[0], fmask[0]);
  puts(dg_last_error(ctx));
  if (dg_destroy(ctx) != DG_OK) return 10;
  return 0;
}
"""


def test_header_is_c99_and_a_c_program_drives_the_library(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = B.load()                                   # builds the library if needed
    libdir = Path(lib._name).resolve().parent
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", str(ROOT / "include"),
                    str(src), "-L", str(libdir), "-ldgeuler", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stderr)
    nums, msg = out.stdout.splitlines()[:2]
    nq, nfq, r0, f0 = nums.split()
    assert (int(nq), int(nfq)) == (27, 9)                   # (p+1)^3 and (p+1)^2 points at p = 2
    assert float(r0) == -1.0 and int(f0) == 0               # node 0 is the vertex (-1,-1,-1), on face 0
    assert msg                                              # the refused step left its reason
