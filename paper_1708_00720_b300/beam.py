"""Binding of the 4+4-bit beamformer (libxengine.so, xe_beam_*).  Argument
marshalling only; the weight conversion and the beamforming run in the
library's CUDA kernels."""
from __future__ import annotations

import ctypes

import torch

from . import xengine as _xe

_P, _I = ctypes.c_void_p, ctypes.c_int
_lib = _xe.library()
for _name, (_args, _res) in {
    "xe_beam_create": ([ctypes.POINTER(_P), _I, _I, _I, _I], _I),
    "xe_beam_destroy": ([_P], _I),
    "xe_beam_set_weights": ([_P, _P, _P], _I),
    "xe_beam_form": ([_P, _P, _I, _P, _P], _I),
    "xe_beam_check": ([_P], _I),
    "xe_beam_last_error": ([_P], ctypes.c_char_p),
}.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


class Beamformer:
    """y[t][c][b] = sum_i w[c][b][i] x[t][c][i] for 4+4-bit gulps [T][C][N]."""

    def __init__(self, n_input: int, n_chan: int, n_beam: int, max_ntime: int):
        self.n_input, self.n_chan, self.n_beam, self.max_ntime = n_input, n_chan, n_beam, max_ntime
        h = _P()
        self._check(_lib.xe_beam_create(ctypes.byref(h), n_input, n_chan, n_beam, max_ntime), "xe_beam_create")
        self.handle = h

    def _check(self, st: int, where: str) -> None:
        if st != _xe.XE_OK:
            h = getattr(self, "handle", None)
            raise _xe.XEngineError(st, where, _lib.xe_beam_last_error(h).decode() if h else "")

    def set_weights(self, w: torch.Tensor, stream=None) -> None:
        """w: complex64 [C][B][N] on the device."""
        if w.dtype != torch.complex64 or tuple(w.shape) != (self.n_chan, self.n_beam, self.n_input):
            raise ValueError(f"weights must be complex64 [{self.n_chan}][{self.n_beam}][{self.n_input}]")
        w = w.contiguous()
        self._w = w                                   # kept alive until the conversion has run
        self._check(_lib.xe_beam_set_weights(self.handle, torch.view_as_real(w).data_ptr(), _xe._stream(stream)),
                    "xe_beam_set_weights")

    def form(self, gulp: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """gulp: uint8 [T][C][N] on the device -> complex64 [T][C][B]."""
        if gulp.dtype != torch.uint8 or gulp.dim() != 3 or not gulp.is_contiguous() or \
                gulp.shape[1] != self.n_chan or gulp.shape[2] != self.n_input:
            raise ValueError("gulp must be a contiguous uint8 tensor [T][C][N]")
        T = gulp.shape[0]
        if out is None:
            out = torch.empty((T, self.n_chan, self.n_beam), dtype=torch.complex64, device=gulp.device)
        self._check(_lib.xe_beam_form(self.handle, gulp.data_ptr() if T else None, T,
                                      torch.view_as_real(out).data_ptr() if T else None, _xe._stream(stream)),
                    "xe_beam_form")
        return out

    def check(self) -> None:
        self._check(_lib.xe_beam_check(self.handle), "xe_beam_check")

    def close(self) -> None:
        if self.handle is not None:
            _lib.xe_beam_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
