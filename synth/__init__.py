"""Seeded synthetic inputs shared by the oracle side and the GPU side.

This module only draws random numbers and writes them in the F-engine's
sample format; it holds none of the X-engine's arithmetic (no unpacking, no
products, no accumulation).  Both the tests and the benchmark feed the same
bytes from here to the CPU oracle and to the CUDA library.

Recipe (stand-in for LWA-SV F-engine output, which is not available here):

* every complex sample has real and imaginary parts drawn from N(0, sigma^2)
  with sigma = 2;
* a common tone of amplitude 3 and frequency 0.05 cycles/sample is added to
  every input of one channel (channel 10 by default), with per-input phase
  phi_i = 0 or phi_i ~ U[0, 2 pi);
* both parts are rounded half-to-even, clipped to [-8, 7] and stored as one
  byte: real part in the high nibble, imaginary part in the low nibble, each
  as 4-bit two's complement (section "Packet capture implementation");
* the layout is uint8[T][C][N] -- time slowest, input fastest -- as the
  capture block delivers a gulp of packets (channels x inputs per time).

Time is drawn in blocks of ``_TBLOCK`` rows, each from its own child of
``numpy.random.SeedSequence(seed)``, so the result is identical whatever the
number of worker threads.
"""
from __future__ import annotations

import hashlib
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_TBLOCK = 64


def _nibble(v: np.ndarray) -> np.ndarray:
    """int in [-8, 7] -> its 4-bit two's-complement code (0..15)."""
    return (v.astype(np.int16) & 0xF).astype(np.uint8)


def pack(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Encode integer parts in [-8, 7] as 4+4-bit bytes (re high, im low)."""
    re = np.asarray(re)
    im = np.asarray(im)
    if re.shape != im.shape:
        raise ValueError("re and im must have the same shape")
    if re.size and (re.min() < -8 or re.max() > 7 or im.min() < -8 or im.max() > 7):
        raise ValueError("components must lie in [-8, 7]")
    return (_nibble(re) << 4) | _nibble(im)


def _phases(seed: int, ninput: int, random_phase: bool) -> np.ndarray:
    if not random_phase:
        return np.zeros(ninput, dtype=np.float64)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x70A5E]))
    return rng.uniform(0.0, 2.0 * np.pi, size=ninput)


def voltages(ninput: int, nchan: int, ntime: int, seed: int, *,
             sigma: float = 2.0, tone_chan: int | None = 10,
             tone_amp: float = 3.0, tone_freq: float = 0.05,
             random_phase: bool = False, threads: int | None = None,
             t0: int = 0) -> np.ndarray:
    """One gulp of 4+4-bit voltages, uint8[ntime][nchan][ninput].

    ``t0`` offsets the time index of the tone, so consecutive gulps of a
    stream continue the same sinusoid.
    """
    if min(ninput, nchan, ntime) < 0:
        raise ValueError("sizes must be non-negative")
    out = np.empty((ntime, nchan, ninput), dtype=np.uint8)
    if out.size == 0:
        return out
    phi = _phases(seed, ninput, random_phase)
    nblk = (ntime + _TBLOCK - 1) // _TBLOCK
    children = np.random.SeedSequence([seed, t0]).spawn(nblk)
    use_tone = tone_chan is not None and 0 <= tone_chan < nchan and tone_amp != 0

    def fill(b: int) -> None:
        ta, tb = b * _TBLOCK, min(ntime, (b + 1) * _TBLOCK)
        rng = np.random.default_rng(children[b])
        shape = (tb - ta, nchan, ninput)
        re = rng.standard_normal(shape, dtype=np.float32) * np.float32(sigma)
        im = rng.standard_normal(shape, dtype=np.float32) * np.float32(sigma)
        if use_tone:
            t = np.arange(ta + t0, tb + t0, dtype=np.float64)[:, None]
            ang = 2.0 * np.pi * tone_freq * t + phi[None, :]
            re[:, tone_chan, :] += (tone_amp * np.cos(ang)).astype(np.float32)
            im[:, tone_chan, :] += (tone_amp * np.sin(ang)).astype(np.float32)
        rq = np.clip(np.rint(re), -8, 7).astype(np.int8)
        iq = np.clip(np.rint(im), -8, 7).astype(np.int8)
        out[ta:tb] = (_nibble(rq) << 4) | _nibble(iq)

    if threads is None:
        threads = min(32, len(os.sched_getaffinity(0)))
    if threads <= 1 or nblk == 1:
        for b in range(nblk):
            fill(b)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(fill, range(nblk)))
    return out


def uniform_bytes(shape, seed: int) -> np.ndarray:
    """Uniformly random packed bytes (every nibble value equally likely)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=shape, dtype=np.uint8)


def sha256(x: np.ndarray) -> str:
    """Content hash of an input array, for caching oracle results."""
    return hashlib.sha256(np.ascontiguousarray(x).tobytes()).hexdigest()


# Workloads (N inputs, C channels, T samples per integration), with the seed
# and phase rule of each.
CONFIGS = {
    "tiny": dict(ninput=16, nchan=64, ntime=1024, seed=1, random_phase=False),
    "lwa": dict(ninput=512, nchan=256, ntime=8192, seed=2, random_phase=True),
    "large_n": dict(ninput=2048, nchan=64, ntime=4096, seed=3, random_phase=True),
}


def config_voltages(name: str, **overrides) -> np.ndarray:
    kw = dict(CONFIGS[name])
    kw.update(overrides)
    return voltages(**kw)


# ---------------------------------------------------------------------------
# gain-calibration inputs
def gains(n_input: int, n_chan: int, seed: int, scatter: float = 0.1) -> np.ndarray:
    """Complex gains g = 1 + scatter * CN(0, 1) per input and channel, [C][N]."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x6A1]))
    z = (rng.standard_normal((n_chan, n_input)) + 1j * rng.standard_normal((n_chan, n_input))) / np.sqrt(2)
    return 1.0 + scatter * z


def sky_model(n_input: int, n_chan: int, seed: int, n_sources: int = 5,
              f_lo: float = 10e6, f_hi: float = 88e6) -> np.ndarray:
    """Model visibilities of a random sky of point sources seen by an
    LWA-SV-like station (section "LWA Sevilleta implementation": dipoles over
    a 100 m x 110 m area, 10-88 MHz).  Input k is polarisation k % 2 of
    antenna k // 2 and both polarisations share the antenna's position.
    Fluxes U[1, 10], directions uniform in the unit disk, channels evenly
    spaced in [f_lo, f_hi].  Returns complex128 [C][N(N+1)/2], packed lower
    triangle: C_ij = sum_s S_s exp(-2 pi i nu/c ((x_i - x_j) l_s + (y_i - y_j) m_s))."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5C1]))
    n_ant = (n_input + 1) // 2
    x = rng.uniform(0.0, 100.0, n_ant)
    y = rng.uniform(0.0, 110.0, n_ant)
    flux = rng.uniform(1.0, 10.0, n_sources)
    rad = np.sqrt(rng.uniform(0.0, 1.0, n_sources))
    ang = rng.uniform(0.0, 2 * np.pi, n_sources)
    l, m = rad * np.cos(ang), rad * np.sin(ang)
    ant = np.arange(n_input) // 2
    ii, jj = np.tril_indices(n_input)
    dx = x[ant[ii]] - x[ant[jj]]
    dy = y[ant[ii]] - y[ant[jj]]
    nu = np.linspace(f_lo, f_hi, n_chan)
    out = np.zeros((n_chan, len(ii)), dtype=np.complex128)
    for s in range(n_sources):
        phase = -2 * np.pi * (nu[:, None] / 299792458.0) * (dx[None, :] * l[s] + dy[None, :] * m[s])
        out += flux[s] * np.exp(1j * phase)
    return out


CALIB_CONFIG = dict(n_input=512, n_chan=128, ntime=1024, seed=4)


# ---------------------------------------------------------------------------
# streaming-service workload: three independent streams (N inputs, C
# channels), gulps of 1024 samples, rings of 8 gulps, integrations of 8 gulps,
# arriving at the LWA-SV cadence (1024 spectra x 40 us per gulp)
SERVE_STREAMS = [
    dict(ninput=256, nchan=64, seed=5),
    dict(ninput=512, nchan=128, seed=6),
    dict(ninput=1024, nchan=256, seed=7),
]
SERVE_GULP = 1024
SERVE_RING = 8
SERVE_INTEGRATE = 8
SERVE_CADENCE_S = 1024 * 40e-6


# ---------------------------------------------------------------------------
# beamformer weights and workload
def beam_weights(n_input: int, n_chan: int, n_beam: int, seed: int,
                 f_lo: float = 10e6, f_hi: float = 88e6) -> np.ndarray:
    """Phase-only weights steering beams to random directions (l, m) in the
    unit disk for an LWA-SV-like station (dipoles in 100 m x 110 m, both
    polarisations of an antenna at its position), channels evenly spaced in
    [f_lo, f_hi]:  w[c][b][i] = exp(+2 pi i nu_c/c (x_i l_b + y_i m_b)) / N.
    complex64 [C][B][N]."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBEA]))
    n_ant = (n_input + 1) // 2
    x = rng.uniform(0.0, 100.0, n_ant)
    y = rng.uniform(0.0, 110.0, n_ant)
    rad = np.sqrt(rng.uniform(0.0, 1.0, n_beam))
    ang = rng.uniform(0.0, 2 * np.pi, n_beam)
    l, m = rad * np.cos(ang), rad * np.sin(ang)
    ant = np.arange(n_input) // 2
    nu = np.linspace(f_lo, f_hi, n_chan)
    ph = 2 * np.pi * (nu[:, None, None] / 299792458.0) * (x[ant][None, None, :] * l[None, :, None] +
                                                          y[ant][None, None, :] * m[None, :, None])
    return (np.exp(1j * ph) / n_input).astype(np.complex64)


BEAM_CONFIG = dict(ninput=512, nchan=256, ntime=8192, nbeam=16, seed=8)
