"""Gain calibration on emitted visibilities: chi^2 and its hand-written
adjoint (libxengine.so, xe_calib_*), behind torch.autograd.Function.

    r_ij = V_ij - g_i conj(g_j) C_ij,   chi2 = sum_c sum_{i>=j} w_ij |r_ij|^2

``g`` is complex64 [C][N]; ``model`` (C_ij) and ``vobs`` (V_ij) are complex64
[C][N(N+1)/2] in the X-engine's packed-lower-triangle layout; ``w`` is
float32 of the same shape or None.  chi^2 is returned as a float64 scalar
tensor on the device; its gradient with respect to ``g`` follows PyTorch's
convention for complex inputs (d/dRe g + i d/dIm g).  All arithmetic runs in
the CUDA kernels; this module only checks shapes and passes pointers.

When ``g`` requires a gradient, the forward call makes one pass over the
visibilities for chi^2 and the unscaled gradient together, and the backward
call only scales that gradient by the incoming one.
"""
from __future__ import annotations

import ctypes

import torch

from . import xengine as _xe


def _fptr(t: torch.Tensor) -> int:
    if t.is_complex():
        t = torch.view_as_real(t)
    if not t.is_contiguous():
        raise ValueError("calibration inputs must be contiguous")
    if not t.is_cuda:
        raise ValueError("calibration inputs must be CUDA tensors")
    return t.data_ptr()


class Calibrator:
    """Owns one xe_calib object (scratch for n_input x n_chan)."""

    def __init__(self, n_input: int, n_chan: int):
        self.n_input, self.n_chan = n_input, n_chan
        h = ctypes.c_void_p()
        _xe._check(_xe.library().xe_calib_create(ctypes.byref(h), n_input, n_chan), "xe_calib_create")
        self.handle = h

    def _args(self, g, model, vobs, w):
        N, C = self.n_input, self.n_chan
        nbl = N * (N + 1) // 2
        if tuple(g.shape) != (C, N) or g.dtype != torch.complex64:
            raise ValueError(f"g must be complex64 [{C}][{N}]")
        for name, t in (("model", model), ("vobs", vobs)):
            if tuple(t.shape) != (C, nbl) or t.dtype != torch.complex64:
                raise ValueError(f"{name} must be complex64 [{C}][{nbl}]")
        if w is not None and (tuple(w.shape) != (C, nbl) or w.dtype != torch.float32):
            raise ValueError(f"w must be float32 [{C}][{nbl}]")
        return _fptr(g), _fptr(model), _fptr(vobs), (_fptr(w) if w is not None else None)

    def chisq(self, g, model, vobs, w=None, include_autos: bool = True, stream=None) -> torch.Tensor:
        out = torch.empty((), dtype=torch.float64, device=g.device)
        pg, pm, pv, pw = self._args(g, model, vobs, w)
        _xe._check(_xe.library().xe_calib_chisq(self.handle, pg, pm, pv, pw, int(include_autos),
                                                 out.data_ptr(), _xe._stream(stream)), "xe_calib_chisq")
        return out

    def grad(self, g, model, vobs, w=None, include_autos: bool = True, scale=None, stream=None) -> torch.Tensor:
        out = torch.empty_like(g)
        pg, pm, pv, pw = self._args(g, model, vobs, w)
        ps = None
        if scale is not None:
            scale = self._scale(scale)
            ps = scale.data_ptr()
        _xe._check(_xe.library().xe_calib_grad(self.handle, pg, pm, pv, pw, int(include_autos), ps,
                                                _fptr(out), _xe._stream(stream)), "xe_calib_grad")
        return out

    def chisq_grad(self, g, model, vobs, w=None, include_autos: bool = True, stream=None,
                   chi_out=None, grad_out=None):
        """(chi2, unscaled gradient) from one pass; chi_out (float64 scalar) and
        grad_out (like g) may be given to reuse output buffers."""
        chi = torch.empty((), dtype=torch.float64, device=g.device) if chi_out is None else chi_out
        out = torch.empty_like(g) if grad_out is None else grad_out
        if chi.dtype != torch.float64 or chi.numel() != 1 or out.shape != g.shape or out.dtype != g.dtype:
            raise ValueError("chi_out must be one float64 and grad_out shaped like g")
        pg, pm, pv, pw = self._args(g, model, vobs, w)
        _xe._check(_xe.library().xe_calib_chisq_grad(self.handle, pg, pm, pv, pw, int(include_autos),
                                                      chi.data_ptr(), _fptr(out), _xe._stream(stream)),
                   "xe_calib_chisq_grad")
        return chi, out

    def scale(self, grad, scale, stream=None) -> torch.Tensor:
        if tuple(grad.shape) != (self.n_chan, self.n_input) or grad.dtype != torch.complex64:
            raise ValueError(f"grad must be complex64 [{self.n_chan}][{self.n_input}]")
        scale = self._scale(scale)
        out = torch.empty_like(grad)
        _xe._check(_xe.library().xe_calib_scale(self.handle, _fptr(grad), scale.data_ptr(), _fptr(out),
                                                 _xe._stream(stream)), "xe_calib_scale")
        return out

    @staticmethod
    def _scale(scale) -> torch.Tensor:
        if scale.dtype != torch.float64 or scale.numel() != 1 or not scale.is_cuda:
            raise ValueError("scale must be one float64 on the device")
        return scale.contiguous()

    def close(self):
        if self.handle is not None:
            _xe.library().xe_calib_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ChiSq(torch.autograd.Function):
    """chi^2(g) with the adjoint kernel as its backward."""

    @staticmethod
    def forward(ctx, g, model, vobs, w, calibrator: Calibrator, include_autos: bool):
        g = g.contiguous()
        ctx.calibrator = calibrator
        if ctx.needs_input_grad[0]:
            chi, grad = calibrator.chisq_grad(g, model, vobs, w, include_autos)
            ctx.save_for_backward(grad)
            return chi
        return calibrator.chisq(g, model, vobs, w, include_autos)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return ctx.calibrator.scale(grad, grad_out), None, None, None, None, None


def chisq(g, model, vobs, w=None, include_autos: bool = True, calibrator: Calibrator | None = None):
    """Differentiable chi^2 (float64 scalar tensor) of complex64 gains g."""
    if calibrator is None:
        calibrator = Calibrator(g.shape[1], g.shape[0])
    return ChiSq.apply(g, model, vobs, w, calibrator, include_autos)
