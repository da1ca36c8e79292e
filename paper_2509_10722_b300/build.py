"""Build the solver's shared library in-tree for sm_103a (B300): libnum_pmp.so, or with
--debug libnum_pmp_debug.so, whose kernels check every gathered index (PMP_DEBUG_BOUNDS).

    python -m paper_2509_10722_b300.build [--force] [--verbose] [--debug]

nvcc cross-compiles without a GPU.  The library exports exactly the C ABI of
include/num_pmp.h and links the CUDA runtime statically.
"""
from __future__ import annotations

import argparse
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libnum_pmp.so")
LIB_DEBUG = os.path.join(LIBDIR, "libnum_pmp_debug.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=(), debug=False):
    """Compile every .cu of csrc/ into lib/libnum_pmp.so (skipped when up to date); with
    debug=True into lib/libnum_pmp_debug.so with the gather bounds checks compiled in."""
    lib = LIB_DEBUG if debug else LIB
    if debug:
        extra = (*extra, "-DPMP_DEBUG_BOUNDS")
    if not force and not _stale(lib):
        return lib
    os.makedirs(LIBDIR, exist_ok=True)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "--cudart", "static", "-I", INCLUDE,
           "-o", tmp, *sources(), *extra]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--debug", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose, debug=a.debug))
    sys.exit(0)
