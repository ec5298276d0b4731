"""Binding of the streaming X-engine service (libxengine.so, xe_service_*).

Argument marshalling only: rings, dispatch, integration, copies and the
dispatcher thread all live in the C++ library.  A stream's gulps are written
into pinned staging slots (``reserve`` returns a numpy view of one, or
``submit`` copies a gulp in) and committed with increasing sequence numbers;
finished integrations come back from ``poll`` as views of pinned output
buffers, which ``release`` hands back to the service.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import xengine as _xe

XE_SERVICE_DRYRUN = 1
XE_SERVICE_MANUAL = 2
XE_SERVICE_NO_BATCH = 4
XE_FAULT_LAUNCH = 1
XE_FAULT_DROP_GULP = 2

_I, _LL, _D, _P = ctypes.c_int, ctypes.c_longlong, ctypes.c_double, ctypes.c_void_p


class StreamConfig(ctypes.Structure):
    _fields_ = [("n_input", _I), ("n_chan", _I), ("gulp_ntime", _I), ("ring_gulps", _I),
                ("integrate_gulps", _I), ("guaranteed", _I), ("operand", _I), ("out_type", _I)]


class Integration(ctypes.Structure):
    _fields_ = [("stream", _I), ("index", _LL), ("first_seq", _LL), ("gulps", _I), ("skipped", _I),
                ("samples", _LL), ("latency_ms", _D), ("vis", _P), ("vis_bytes", _LL), ("status", _I)]


class StreamStats(ctypes.Structure):
    _fields_ = [("committed", _LL), ("skipped_full", _LL), ("dropped", _LL), ("launches", _LL),
                ("gulps_correlated", _LL), ("integrations", _LL), ("max_batch", _LL),
                ("device_bytes", _LL), ("host_bytes", _LL), ("state", _I), ("pending", _I),
                ("inflight", _I), ("shared_launches", _LL)]


def _setup(lib: ctypes.CDLL) -> None:
    sigs = {
        "xe_service_create": ([ctypes.POINTER(_P), _LL, _I], _I),
        "xe_service_destroy": ([_P], _I),
        "xe_service_add_stream": ([_P, ctypes.POINTER(StreamConfig), ctypes.POINTER(_I)], _I),
        "xe_service_reserve": ([_P, _I, _I, ctypes.POINTER(_P)], _I),
        "xe_service_commit": ([_P, _I, _LL], _I),
        "xe_service_submit": ([_P, _I, _P, _LL, _I], _I),
        "xe_service_flush": ([_P, _I], _I),
        "xe_service_poll": ([_P, _I, _I, ctypes.POINTER(Integration)], _I),
        "xe_service_release": ([_P, _I, _LL], _I),
        "xe_service_stats": ([_P, _I, ctypes.POINTER(StreamStats)], _I),
        "xe_service_inject": ([_P, _I, _I], _I),
        "xe_service_dryrun_complete": ([_P, _I], _I),
        "xe_service_last_error": ([_P], ctypes.c_char_p),
        "xe_wait_flag": ([_P, _I, _LL, _P, _P], _I),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


_lib = _xe.library()
_setup(_lib)


class ServiceError(_xe.XEngineError):
    pass


class Service:
    """One xe_service; streams are added with ``add_stream``."""

    def __init__(self, mem_cap_bytes: int = 0, dryrun: bool = False, manual: bool = False,
                 batch: bool = True):
        flags = ((XE_SERVICE_DRYRUN if dryrun else 0) | (XE_SERVICE_MANUAL if manual else 0) |
                 (0 if batch else XE_SERVICE_NO_BATCH))
        h = _P()
        self._check(_lib.xe_service_create(ctypes.byref(h), int(mem_cap_bytes), flags), "xe_service_create", None)
        self.handle = h
        self.configs: dict[int, StreamConfig] = {}

    @staticmethod
    def _check(status: int, where: str, handle) -> None:
        if status != _xe.XE_OK:
            detail = _lib.xe_service_last_error(handle).decode() if handle else ""
            raise ServiceError(status, where, detail)

    def add_stream(self, n_input: int, n_chan: int, gulp_ntime: int, ring_gulps: int = 8,
                   integrate_gulps: int = 8, guaranteed: bool = True, operand: str = "fp8",
                   out: str = "ci32") -> int:
        cfg = StreamConfig(n_input, n_chan, gulp_ntime, ring_gulps, integrate_gulps, int(guaranteed),
                           _xe.OPERANDS[operand], _xe.XE_OUT_CF32 if out == "cf32" else _xe.XE_OUT_CI32)
        sid = _I()
        self._check(_lib.xe_service_add_stream(self.handle, ctypes.byref(cfg), ctypes.byref(sid)),
                    "xe_service_add_stream", self.handle)
        self.configs[sid.value] = cfg
        return sid.value

    def gulp_shape(self, sid: int) -> tuple[int, int, int]:
        c = self.configs[sid]
        return (c.gulp_ntime, c.n_chan, c.n_input)

    def reserve(self, sid: int, timeout_ms: int = 1000):
        """Numpy view (uint8 [T][C][N]) of the next staging slot, or None if
        the ring is full (XE_ERR_BUSY)."""
        p = _P()
        st = _lib.xe_service_reserve(self.handle, sid, timeout_ms, ctypes.byref(p))
        if st == _xe.XE_ERR_BUSY:
            return None
        self._check(st, "xe_service_reserve", self.handle)
        shape = self.gulp_shape(sid)
        buf = (ctypes.c_uint8 * int(np.prod(shape))).from_address(p.value)
        return np.ctypeslib.as_array(buf).reshape(shape)

    def commit(self, sid: int, seq: int) -> None:
        self._check(_lib.xe_service_commit(self.handle, sid, seq), "xe_service_commit", self.handle)

    def submit(self, sid: int, gulp: np.ndarray, seq: int, timeout_ms: int = 1000) -> bool:
        """Copy one gulp in and commit it; False if the ring was full."""
        if gulp.dtype != np.uint8 or gulp.shape != self.gulp_shape(sid) or not gulp.flags.c_contiguous:
            raise ValueError(f"gulp must be contiguous uint8 {self.gulp_shape(sid)}")
        st = _lib.xe_service_submit(self.handle, sid, gulp.ctypes.data, seq, timeout_ms)
        if st == _xe.XE_ERR_BUSY:
            return False
        self._check(st, "xe_service_submit", self.handle)
        return True

    def flush(self, sid: int) -> None:
        self._check(_lib.xe_service_flush(self.handle, sid), "xe_service_flush", self.handle)

    def poll(self, sid: int, timeout_ms: int = 0):
        """The oldest finished integration as a dict (its 'vis' is a view of
        the pinned output buffer, valid until release), or None."""
        out = Integration()
        st = _lib.xe_service_poll(self.handle, sid, timeout_ms, ctypes.byref(out))
        if st == _xe.XE_ERR_BUSY:
            return None
        self._check(st, "xe_service_poll", self.handle)
        c = self.configs[sid]
        nbl = c.n_input * (c.n_input + 1) // 2
        ctype = ctypes.c_float if c.out_type == _xe.XE_OUT_CF32 else ctypes.c_int32
        buf = (ctype * (out.vis_bytes // 4)).from_address(out.vis)
        vis = np.ctypeslib.as_array(buf).reshape(c.n_chan, nbl, 2)
        return {"stream": out.stream, "index": out.index, "first_seq": out.first_seq, "gulps": out.gulps,
                "skipped": out.skipped, "samples": out.samples, "latency_ms": out.latency_ms,
                "vis": vis, "status": out.status}

    def release(self, sid: int, index: int) -> None:
        self._check(_lib.xe_service_release(self.handle, sid, index), "xe_service_release", self.handle)

    def stats(self, sid: int) -> dict:
        s = StreamStats()
        self._check(_lib.xe_service_stats(self.handle, sid, ctypes.byref(s)), "xe_service_stats", self.handle)
        return {name: getattr(s, name) for name, _ in StreamStats._fields_}

    def inject(self, sid: int, fault: int) -> None:
        self._check(_lib.xe_service_inject(self.handle, sid, fault), "xe_service_inject", self.handle)

    def dryrun_complete(self, sid: int) -> None:
        self._check(_lib.xe_service_dryrun_complete(self.handle, sid), "xe_service_dryrun_complete", self.handle)

    def close(self) -> None:
        if self.handle is not None:
            _lib.xe_service_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def xe_wait_flag(d_flag, expected: int, timeout_ns: int, d_status, stream=None) -> None:
    """Bounded device-side wait (see include/xengine.h); status lands in d_status."""
    st = _lib.xe_wait_flag(_xe._ptr(d_flag), expected, timeout_ns, _xe._ptr(d_status), _xe._stream(stream))
    if st != _xe.XE_OK:
        raise ServiceError(st, "xe_wait_flag")
