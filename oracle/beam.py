"""Phase-and-sum beamformer on 4+4-bit voltages, float64 -- TEST
INFRASTRUCTURE ONLY (the product library never imports it).

The DRX pipeline's beamformer ("LWA Sevilleta implementation") forms beams
directly from the 4+4-bit samples: for every time t, channel c and beam b

    y[t][c][b] = sum_i w[c][b][i] * x[t][c][i]

with complex weights w (a phase per input, optionally an amplitude).  The
GPU path multiplies in float16 on the tensor cores, so the weights enter as
their float16 roundings (real and imaginary parts rounded separately); the
oracle applies the same rounding (`round_weights`) and then evaluates the
definition exactly in complex128.  Pinned in tests/test_beam_oracle.py by a
hand-worked product, identity and linearity cases, a steered tone (closed
form N * s_t), an explicit loop, and binary16 roundings worked out by hand
(ties, subnormals, overflow, parts rounding in different directions:
tests/golden/beam_weight_rounding.txt).

Arrays: x uint8 [T][C][N] (the X-engine's gulp layout, decoded by this
module's own nibble decoder), w complex [C][B][N]; y complex128 [T][C][B].
"""
from __future__ import annotations

import numpy as np


def decode(gulp: np.ndarray) -> np.ndarray:
    """uint8 samples -> complex128: real = high nibble, imaginary = low nibble,
    each 4-bit two's complement."""
    g = np.asarray(gulp, dtype=np.int16)
    re = (g >> 4) & 0xF
    im = g & 0xF
    re = np.where(re >= 8, re - 16, re)
    im = np.where(im >= 8, im - 16, im)
    return re.astype(np.float64) + 1j * im.astype(np.float64)


def round_weights(w: np.ndarray) -> np.ndarray:
    """The operand precision of the GPU path: float16 real and imaginary parts."""
    w = np.asarray(w)
    return (w.real.astype(np.float16).astype(np.float64) +
            1j * w.imag.astype(np.float16).astype(np.float64))


def beamform(gulp: np.ndarray, w: np.ndarray, rounded: bool = True) -> np.ndarray:
    x = decode(gulp)
    ww = round_weights(w) if rounded else np.asarray(w, dtype=np.complex128)
    return np.einsum("tci,cbi->tcb", x, ww)


def beamform_one(gulp, w, t: int, c: int, b: int, rounded: bool = True) -> complex:
    """One output by an explicit sum, for sampled checks at full size."""
    ww = round_weights(w[c, b]) if rounded else np.asarray(w[c, b], dtype=np.complex128)
    x = decode(gulp[t, c])
    total = 0j
    for i in range(x.shape[0]):
        total += ww[i] * x[i]
    return total
