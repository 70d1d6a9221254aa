"""Build the in-tree shared library ``libdgeuler.so`` (sm_103a).

Compiles each translation unit in parallel (g++ for host-only C++, nvcc for
CUDA) into ``_build/`` and links with ``nvcc -shared``. Rebuilds only when a
source or header is newer than the library.

``build(debug=True)`` (``python -m paper_1710_03887_gb300.build_lib --debug``)
makes the debug variant ``libdgeuler_debug.so`` from the same sources with
``-DDG_BOUNDS_CHECK``: every index a kernel reads from the mesh tables is
checked before the access it selects, and a failed check is reported as
DG_ERR_BOUNDS. It is built on demand only, not by the package's build step.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = PKG / "libdgeuler.so"
BUILD_DEBUG = PKG / "_build_debug"
LIB_DEBUG = PKG / "libdgeuler_debug.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CXX_SOURCES = ["operators.cpp", "mesh.cpp", "modal_ops.cpp"]
CU_SOURCES = ["context.cu", "stage_fp64.cu", "stage_f32.cu", "stage_tc.cu", "learned.cu", "totals_static.cu",
              "stage_modal.cu", "halo.cu", "closure_tc.cu"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libdgeuler.so")


def _inputs():
    files = [CSRC / s for s in CXX_SOURCES + CU_SOURCES]
    files += list(CSRC.glob("*.hpp")) + list(CSRC.glob("*.cuh")) + list((ROOT / "include").glob("*.h"))
    files.append(Path(__file__))
    return files


def up_to_date(debug=False):
    lib = LIB_DEBUG if debug else LIB
    if not lib.exists():
        return False
    t = lib.stat().st_mtime
    return all(f.stat().st_mtime <= t for f in _inputs())


def build(force=False, verbose=False, debug=False):
    """Compile and link; returns the library path (the debug variant with
    ``debug``)."""
    lib, bdir = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if not force and up_to_date(debug):
        return lib
    nvcc = _nvcc()
    bdir.mkdir(exist_ok=True)
    flags = ["-DDG_BOUNDS_CHECK"] if debug else []
    inc = ["-I", str(ROOT / "include"), "-I", str(CSRC)]
    jobs = []
    objs = []
    for s in CXX_SOURCES:
        o = bdir / (s + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", *flags, *inc, "-c", str(CSRC / s), "-o",
               str(o)]
        jobs.append((s, cmd))
        objs.append(o)
    for s in CU_SOURCES:
        o = bdir / (s + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xptxas", "-warn-spills", *flags, *inc, "-c", str(CSRC / s), "-o", str(o)]
        jobs.append((s, cmd))
        objs.append(o)
    procs = [(s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
             for s, cmd in jobs]
    failed = []
    for s, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed.append((s, out))
    if failed:
        msg = "\n".join(f"--- {s}\n{out}" for s, out in failed)
        raise RuntimeError(f"compilation failed:\n{msg}")
    tmp = lib.with_suffix(".so.tmp")
    link = [nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
