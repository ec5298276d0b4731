"""CPU oracle for the X-engine -- TEST INFRASTRUCTURE ONLY.

The oracle is the plain, slow, obviously correct definition of what the GPU
path computes.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product library never imports, links or executes anything here, and this
package imports nothing from the product package.

Functions
---------
* :func:`decode` / :func:`unpack` -- the 4+4-bit complex sample format of the
  paper's section "Packet capture implementation" (signed 4-bit real part in
  the high nibble, signed 4-bit imaginary part in the low nibble), widened to
  8+8 bits as the TBN pipeline's unpack stage does.
* :func:`correlate` -- the X-engine itself: per channel, the Hermitian
  visibility matrix V_c = sum_t x_t x_t^H, packed lower triangle, exact int64
  (the linear-algebra module of section "Back end", fed by the unpack block of
  section "Some included blocks").
* :func:`correlate_one` -- one visibility, for sampled checks at full size.
* :mod:`oracle.calib` -- the gain-calibration chi^2 and its gradient in fp64.
* :mod:`oracle.beamform` -- the phase-and-sum beam of section "DRX Pipeline".

Parity is pinned in ``tests/test_oracle.py`` (see the C file's header).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xcorr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O3 -march=native, no hand SIMD)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O3", "-march=native", "-std=c11", "-fPIC", "-shared",
             "-pthread", "-Wall", "-Wextra", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, p = ctypes.c_int64, ctypes.c_void_p
            lib.oracle_correlate.argtypes = [p, i64, i64, i64, p, ctypes.c_int,
                                             ctypes.c_int]
            lib.oracle_correlate.restype = ctypes.c_int
            lib.oracle_correlate_one.argtypes = [p, i64, i64, i64, i64, i64,
                                                 i64, p, p]
            lib.oracle_correlate_one.restype = None
            lib.oracle_unpack.argtypes = [p, ctypes.c_size_t, p]
            lib.oracle_unpack.restype = None
            lib.oracle_decode_byte.argtypes = [ctypes.c_uint8, p, p]
            lib.oracle_decode_byte.restype = None
            _lib = lib
    return _lib


def default_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def decode(b: int) -> tuple[int, int]:
    """(re, im) of one packed byte."""
    lib = _load()
    re, im = ctypes.c_int(), ctypes.c_int()
    lib.oracle_decode_byte(ctypes.c_uint8(b), ctypes.byref(re), ctypes.byref(im))
    return re.value, im.value


def unpack(packed: np.ndarray) -> np.ndarray:
    """uint8[...] -> int8[..., 2] (re, im)."""
    x = np.ascontiguousarray(packed, dtype=np.uint8)
    out = np.empty(x.shape + (2,), dtype=np.int8)
    _load().oracle_unpack(x.ctypes.data, x.size, out.ctypes.data)
    return out


def correlate(x: np.ndarray, full_square: bool = False,
              nthreads: int | None = None) -> np.ndarray:
    """Exact visibilities of one gulp.

    x: uint8[T][C][N].  Returns int64[C][N(N+1)/2][2] (packed lower triangle,
    index i(i+1)/2 + j for i >= j) or, with ``full_square``, int64[C][N][N][2]
    holding every ordered pair.
    """
    x = np.ascontiguousarray(x, dtype=np.uint8)
    if x.ndim != 3:
        raise ValueError("x must be uint8[T][C][N]")
    T, C, N = x.shape
    nbl = N * N if full_square else N * (N + 1) // 2
    out = np.zeros((C, nbl, 2), dtype=np.int64)
    if nthreads is None:
        nthreads = default_threads()
    rc = _load().oracle_correlate(x.ctypes.data, T, C, N, out.ctypes.data,
                                  int(full_square), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_correlate rejected its arguments")
    if full_square:
        out = out.reshape(C, N, N, 2)
    return out


def correlate_one(x: np.ndarray, c: int, i: int, j: int) -> tuple[int, int]:
    """Exact V_c[i][j] (any ordered pair) of one gulp x: uint8[T][C][N]."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    T, C, N = x.shape
    if not (0 <= c < C and 0 <= i < N and 0 <= j < N):
        raise IndexError("visibility index out of range")
    re, im = ctypes.c_int64(), ctypes.c_int64()
    _load().oracle_correlate_one(x.ctypes.data, T, C, N, c, i, j,
                                 ctypes.byref(re), ctypes.byref(im))
    return re.value, im.value


def tri_index(i: int, j: int) -> int:
    """Packed lower-triangle position of baseline (i, j), i >= j."""
    return i * (i + 1) // 2 + j
