"""Build the X-engine shared library (libxengine.so) in-tree for sm_103a.

nvcc cross-compiles without a GPU.  The library links the CUDA runtime
statically and resolves driver entry points at run time, so it loads on a
machine without a GPU driver (its calls then return an error).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libxengine.so")
# The same sources with XE_DEBUG_CHECKS: every global store of the X-engine
# kernels is index-checked against its buffer (a skipped access sets an
# error bit instead of faulting); used by the tests as a memory checker.
LIB_DEBUG = os.path.join(HERE, "libxengine_debug.so")
ROOT = os.path.dirname(HERE)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-shared", "-cudart", "static", "-Xptxas", "-v"]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        sorted(glob.glob(os.path.join(CSRC, "*.h"))) + [os.path.join(ROOT, "include", "xengine.h")]


def is_stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and not is_stale(lib):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    extra = ["-DXE_DEBUG_CHECKS"] if debug else []
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-o", tmp, *sources()]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError(f"nvcc failed building {os.path.basename(lib)}")
    if verbose:
        sys.stderr.write(res.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
    if "--debug" in sys.argv:
        build(force="--force" in sys.argv, debug=True)
        print(LIB_DEBUG)
