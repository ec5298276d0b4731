"""Python binding of the X-engine C ABI (include/xengine.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``libxengine.so``.  Functions keep the C names; tensors are passed
as raw device pointers (``Tensor.data_ptr()``) and streams as
``torch.cuda.Stream.cuda_stream`` (default: torch's current stream).  A
non-OK status raises :class:`XEngineError`.

There is no CPU fallback: if the library cannot be loaded, importing this
module raises.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

XE_OK = 0
XE_ERR_INVALID_ARG = 1
XE_ERR_ALIGNMENT = 2
XE_ERR_SHAPE = 3
XE_ERR_ACCUM_BOUND = 4
XE_ERR_NOMEM = 5
XE_ERR_CUDA = 6
XE_ERR_DEVICE_UNSUPPORTED = 7
XE_ERR_TIMEOUT = 8
XE_ERR_BUSY = 9
XE_ERR_DEVICE_INDEX = 10

XE_OPERAND_FP8_E4M3 = 0
XE_OPERAND_FP16 = 1
XE_OPERAND_INT32_CUDACORE = 2

XE_OUT_CI32 = 0
XE_OUT_CF32 = 1

XE_MAX_SAMPLES_CI32 = 16777215
XE_MAX_SAMPLES_CF32 = 131072

OPERANDS = {"fp8": XE_OPERAND_FP8_E4M3, "fp16": XE_OPERAND_FP16,
            "int32": XE_OPERAND_INT32_CUDACORE}


class XEngineError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {xe_status_string(status)} (status {status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def _load(debug: bool = False) -> ctypes.CDLL:
    path = _build.LIB_DEBUG if debug else _build.LIB
    if not os.path.exists(path) or _build.is_stale(path):
        _build.build(debug=debug)
    lib = ctypes.CDLL(path)
    P, I, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    sigs = {
        "xe_plan_create": ([ctypes.POINTER(P), I, I, I, I, I], I),
        "xe_plan_destroy": ([P], I),
        "xe_unpack": ([P, P, P, I, P], I),
        "xe_correlate": ([P, P, I, I, P], I),
        "xe_integrate": ([P, P, P], I),
        "xe_correlate_emit": ([P, P, I, P, P], I),
        "xe_reset": ([P, P], I),
        "xe_samples_integrated": ([P, ctypes.POINTER(LL)], I),
        "xe_correlate_host": ([P, P, I, I, P], I),
        "xe_plan_check": ([P], I),
        "xe_plan_launch_count": ([P, ctypes.POINTER(LL)], I),
        "xe_calib_create": ([ctypes.POINTER(P), I, I], I),
        "xe_calib_destroy": ([P], I),
        "xe_calib_chisq": ([P, P, P, P, P, I, P, P], I),
        "xe_calib_grad": ([P, P, P, P, P, I, P, P, P], I),
        "xe_calib_chisq_grad": ([P, P, P, P, P, I, P, P, P], I),
        "xe_calib_scale": ([P, P, P, P, P], I),
        "xe_status_string": ([I], ctypes.c_char_p),
        "xe_plan_last_error": ([P], ctypes.c_char_p),
        "xe_version": ([], ctypes.c_char_p),
        "xe_probe_dp4a_rate": ([I, I, P, P, ctypes.POINTER(LL), P], I),
        "xe_correlate_batch": ([I, P, P, P, P, P], I),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()
LIBRARY_PATH = _build.LIB


def header_functions() -> list[str]:
    """Names of the functions include/xengine.h declares."""
    hdr = os.path.join(os.path.dirname(_build.HERE), "include", "xengine.h")
    return re.findall(r"^XE_API\s+[\w\s\*]+?\b(xe_\w+)\s*\(", open(hdr).read(), flags=re.M)


def library() -> ctypes.CDLL:
    return _lib


_debug_lib = None


def debug_library() -> ctypes.CDLL:
    """The index-checked build (XE_DEBUG_CHECKS) of the same library, loaded
    beside the normal one: its X-engine kernels check every global store
    against its buffer and report a miss through xe_plan_check as
    XE_ERR_DEVICE_INDEX instead of writing outside it."""
    global _debug_lib
    if _debug_lib is None:
        _debug_lib = _load(debug=True)
    return _debug_lib


def xe_status_string(status: int) -> str:
    return _lib.xe_status_string(int(status)).decode()


def xe_version() -> str:
    return _lib.xe_version().decode()


def _ptr(x) -> int | None:
    """Device/host pointer of a tensor, numpy array or integer address."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, where: str, plan=None) -> None:
    if status != XE_OK:
        detail = _lib.xe_plan_last_error(plan).decode() if plan else ""
        raise XEngineError(status, where, detail)


def xe_plan_create(n_input: int, n_chan: int, max_ntime: int,
                   op: int = XE_OPERAND_FP8_E4M3, out_type: int = XE_OUT_CI32):
    """Returns an opaque plan handle (ctypes.c_void_p)."""
    plan = ctypes.c_void_p()
    _check(_lib.xe_plan_create(ctypes.byref(plan), n_input, n_chan, max_ntime, op, out_type),
           "xe_plan_create")
    return plan


def xe_plan_destroy(plan) -> None:
    _check(_lib.xe_plan_destroy(plan), "xe_plan_destroy")


def xe_unpack(plan, d_packed, d_ci8, ntime: int, stream=None) -> None:
    _check(_lib.xe_unpack(plan, _ptr(d_packed), _ptr(d_ci8), ntime, _stream(stream)),
           "xe_unpack", plan)


def xe_correlate(plan, d_gulp, ntime: int, accumulate: int = 0, stream=None) -> None:
    _check(_lib.xe_correlate(plan, _ptr(d_gulp), ntime, accumulate, _stream(stream)),
           "xe_correlate", plan)


def xe_correlate_batch(plans, gulps, ntimes, accumulates, stream=None) -> None:
    """One launch correlating gulps[k] (ntimes[k] samples) into plans[k]."""
    n = len(plans)
    arr_p = (ctypes.c_void_p * n)(*plans)
    arr_g = (ctypes.c_void_p * n)(*[_ptr(g) for g in gulps])
    arr_t = (ctypes.c_int * n)(*[int(t) for t in ntimes])
    arr_a = (ctypes.c_int * n)(*[int(a) for a in accumulates])
    _check(_lib.xe_correlate_batch(n, arr_p, arr_g, arr_t, arr_a, _stream(stream)), "xe_correlate_batch",
           plans[0] if n else None)


def xe_integrate(plan, d_vis, stream=None) -> None:
    _check(_lib.xe_integrate(plan, _ptr(d_vis), _stream(stream)), "xe_integrate", plan)


def xe_correlate_emit(plan, d_gulp, ntime: int, d_vis, stream=None) -> None:
    _check(_lib.xe_correlate_emit(plan, _ptr(d_gulp), ntime, _ptr(d_vis), _stream(stream)),
           "xe_correlate_emit", plan)


def xe_reset(plan, stream=None) -> None:
    _check(_lib.xe_reset(plan, _stream(stream)), "xe_reset", plan)


def xe_samples_integrated(plan) -> int:
    out = ctypes.c_longlong()
    _check(_lib.xe_samples_integrated(plan, ctypes.byref(out)), "xe_samples_integrated")
    return out.value


def xe_correlate_host(plan, h_gulp, ntime: int, accumulate: int, h_vis) -> None:
    _check(_lib.xe_correlate_host(plan, _ptr(h_gulp), ntime, accumulate, _ptr(h_vis)),
           "xe_correlate_host", plan)


def xe_plan_check(plan) -> None:
    _check(_lib.xe_plan_check(plan), "xe_plan_check", plan)


def xe_plan_launch_count(plan) -> int:
    out = ctypes.c_longlong()
    _check(_lib.xe_plan_launch_count(plan, ctypes.byref(out)), "xe_plan_launch_count")
    return out.value


def dp4a_rate_per_sm_clock(device=None, iters: int = 4096) -> float:
    """Measured dp4a issue rate of the CUDA cores: dp4a per SM per clock
    (the arithmetic ceiling of the plain int32 X-engine)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    ctas = torch.cuda.get_device_properties(dev).multi_processor_count   # one CTA per SM
    cycles = torch.zeros(ctas, dtype=torch.int64, device=dev)
    sink = torch.zeros(ctas * 256, dtype=torch.int32, device=dev)
    per = ctypes.c_longlong()
    for _ in range(2):                   # the first launch warms up
        _check(_lib.xe_probe_dp4a_rate(iters, ctas, cycles.data_ptr(), sink.data_ptr(),
                                       ctypes.byref(per), _stream(None)), "xe_probe_dp4a_rate")
    torch.cuda.synchronize(dev)
    # each SM ran one CTA: its rate is that CTA's dp4a over its span
    return per.value / float(cycles.double().median())


def status_of(fn, *args) -> int:
    """Call a raw C entry point and return its status instead of raising."""
    return getattr(_lib, fn)(*args)


class XEngine:
    """Convenience owner of one plan (same calls, torch tensors in and out)."""

    def __init__(self, n_input: int, n_chan: int, max_ntime: int, operand: str = "fp8",
                 out: str = "ci32"):
        import torch
        self.n_input, self.n_chan, self.max_ntime = n_input, n_chan, max_ntime
        self.operand = operand
        self.out = out
        self._torch = torch
        self.plan = xe_plan_create(n_input, n_chan, max_ntime, OPERANDS[operand],
                                   XE_OUT_CF32 if out == "cf32" else XE_OUT_CI32)

    @property
    def n_baselines(self) -> int:
        return self.n_input * (self.n_input + 1) // 2

    def vis_empty(self, device="cuda", pin_memory=False):
        dt = self._torch.float32 if self.out == "cf32" else self._torch.int32
        return self._torch.empty((self.n_chan, self.n_baselines, 2), dtype=dt, device=device,
                                 pin_memory=pin_memory)

    def correlate(self, gulp, accumulate: bool = False, stream=None) -> None:
        if gulp.dtype != self._torch.uint8 or gulp.dim() != 3 or not gulp.is_contiguous():
            raise ValueError("gulp must be a contiguous uint8 tensor [T][C][N]")
        if gulp.shape[1] != self.n_chan or gulp.shape[2] != self.n_input:
            raise ValueError("gulp shape does not match the plan")
        xe_correlate(self.plan, gulp, gulp.shape[0], int(accumulate), stream)

    def integrate(self, out=None, stream=None):
        if out is None:
            out = self.vis_empty(device="cuda")
        xe_integrate(self.plan, out, stream)
        return out

    def correlate_emit(self, gulp, out=None, stream=None):
        """Visibilities of this gulp alone, written straight into `out`
        (ci32 plans); the plan's accumulator is not touched."""
        if gulp.dtype != self._torch.uint8 or gulp.dim() != 3 or not gulp.is_contiguous():
            raise ValueError("gulp must be a contiguous uint8 tensor [T][C][N]")
        if gulp.shape[1] != self.n_chan or gulp.shape[2] != self.n_input:
            raise ValueError("gulp shape does not match the plan")
        if out is None:
            out = self.vis_empty(device="cuda")
        xe_correlate_emit(self.plan, gulp, gulp.shape[0], out, stream)
        return out

    def reset(self, stream=None) -> None:
        xe_reset(self.plan, stream)

    def samples(self) -> int:
        return xe_samples_integrated(self.plan)

    def check(self) -> None:
        xe_plan_check(self.plan)

    def close(self) -> None:
        if self.plan is not None:
            xe_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
