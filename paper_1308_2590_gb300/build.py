"""Build libpic.so (the CUDA library behind include/pic.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
paper_1308_2590_gb300/_build/libpic.so.  Run as a module or call build().
build(checks=True) makes _build/checks/libpic_checks.so instead: the same
sources with PIC_CHECKS defined, whose kernels test their invariants (indices
in range, offsets in [0, 1), shared-memory canaries) and report a broken one
as an error instead of touching memory out of range.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpic.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-I" + os.path.join(HERE, "..", "include"), "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(HERE, "..", "include", "*.h")))


CHECKS_OUT = os.path.join(OUT, "checks")
CHECKS_LIB = os.path.join(CHECKS_OUT, "libpic_checks.so")


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _sources() + _headers())


def _compile(src: str, verbose: bool, out: str = OUT, extra=()) -> str:
    obj = os.path.join(out, os.path.basename(src).replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link libpic.so (libpic_checks.so
    with checks=True); returns its path."""
    out, lib = (CHECKS_OUT, CHECKS_LIB) if checks else (OUT, LIB)
    extra = ("-DPIC_CHECKS",) if checks else ()
    os.makedirs(out, exist_ok=True)
    if not force and not _stale(lib):
        return lib
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, out, extra), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checks="--checks" in sys.argv))
