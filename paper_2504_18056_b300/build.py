"""Build libgmcs.so (the C-ABI library of include/gmcs.h) and libgmcs_diag.so
(the diagnostics of include/gmcs_diag.h) in-tree for sm_103a.

    python -m paper_2504_18056_b300.build [--force] [--verbose]

Each .cu under csrc/ (csrc/diag/ for the diagnostics) is compiled to an object
with nvcc and the objects are linked into a shared library next to this file.
--verbose adds -Xptxas -v (register / spill / shared-memory report per kernel).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libgmcs.so")
DIAG_OUT = os.path.join(HERE, "libgmcs_diag.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def sources(diag=False):
    return sorted(glob.glob(os.path.join(CSRC, "diag", "*.cu") if diag else os.path.join(CSRC, "*.cu")))


def _stale(out, diag):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = sources(diag) + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def _link(out, diag, verbose):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    for src in sources(diag):
        obj = os.path.join(BUILD, ("diag_" if diag else "") + os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
        subprocess.run(cmd, check=True)
        objs.append(obj)
    tmp = out + ".tmp"
    subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], check=True)
    os.replace(tmp, out)


def build(force=False, verbose=False):
    """Build both libraries if a source is newer; returns the path of libgmcs.so."""
    for out, diag in ((OUT, False), (DIAG_OUT, True)):
        if force or _stale(out, diag):
            _link(out, diag, verbose)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
