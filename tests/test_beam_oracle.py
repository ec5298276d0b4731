"""Pins for the float64 beamformer oracle (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import beam


def test_hand_worked_product():
    # byte 0x7F = 7 - 1i; w = 1 + 2i: (7 - i)(1 + 2i) = 7 + 14i - i + 2 = 9 + 13i
    g = np.array([[[0x7F]]], np.uint8)
    w = np.array([[[1 + 2j]]], np.complex64)
    assert beam.beamform(g, w)[0, 0, 0] == 9 + 13j


def test_decoder_corners():
    g = np.array([[[0x80, 0x0F, 0x77, 0x88]]], np.uint8)
    np.testing.assert_array_equal(beam.decode(g)[0, 0], [-8 + 0j, 0 - 1j, 7 + 7j, -8 - 8j])


def test_identity_beam_returns_the_input():
    rng = np.random.default_rng(0)
    g = rng.integers(0, 256, (5, 3, 7), dtype=np.uint8)
    w = np.zeros((3, 7, 7), np.complex64)
    for i in range(7):
        w[:, i, i] = 1
    np.testing.assert_array_equal(beam.beamform(g, w), beam.decode(g))


def test_linearity_in_the_weights():
    rng = np.random.default_rng(1)
    g = rng.integers(0, 256, (4, 2, 9), dtype=np.uint8)
    w1 = synth.beam_weights(9, 2, 3, 1).astype(np.complex128) * 9
    w2 = synth.beam_weights(9, 2, 3, 2).astype(np.complex128) * 9
    a = beam.beamform(g, w1, rounded=False) + 2 * beam.beamform(g, w2, rounded=False)
    np.testing.assert_allclose(beam.beamform(g, w1 + 2 * w2, rounded=False), a, rtol=1e-12, atol=1e-9)


def test_steered_tone_sums_coherently():
    # x[t][i] = s_t e^{i phi_i} exactly representable: phases multiples of pi/2
    rng = np.random.default_rng(2)
    T, N = 16, 12
    s = rng.integers(-7, 8, T)
    k = rng.integers(0, 4, N)
    u = np.array([1, 1j, -1, -1j])[k]
    x = s[:, None] * u[None, :]
    g = synth.pack(x.real.astype(int), x.imag.astype(int))[:, None, :]
    w = np.conj(u)[None, None, :].astype(np.complex64)          # steer onto the tone
    y = beam.beamform(g, w)[:, 0, 0]
    np.testing.assert_array_equal(y, N * s)


def test_explicit_loop_matches_einsum_and_rounding_is_float16():
    rng = np.random.default_rng(3)
    g = rng.integers(0, 256, (3, 2, 11), dtype=np.uint8)
    w = synth.beam_weights(11, 2, 4, 3) * 7.3
    y = beam.beamform(g, w)
    for t in range(3):
        for c in range(2):
            for b in range(4):
                assert abs(beam.beamform_one(g, w, t, c, b) - y[t, c, b]) < 1e-12
    wr = beam.round_weights(w)
    assert np.all(wr.real == w.real.astype(np.float16).astype(np.float64))
    assert np.abs(wr - w).max() <= 2.0 ** -11 * np.abs(w).max() * 2


def _rounding_cases():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "beam_weight_rounding.txt")
    rows = []
    with open(path) as f:
        for line in f:
            body = line.split("#", 1)[0].split()
            if body:
                rows.append([float(v) for v in body])
    a = np.array(rows)
    return a[:, 0] + 1j * a[:, 1], a[:, 2], a[:, 3]


def _rtz16(x):
    """Binary16 with truncation toward zero (a wrong reading, for the teeth check)."""
    with np.errstate(over="ignore"):
        r = x.astype(np.float16).astype(np.float64)
    over = np.abs(r) > np.abs(x)
    r[over] = np.nextafter(r[over].astype(np.float16), np.float16(0)).astype(np.float64)
    return r


def _bf16(x):
    """bfloat16, round to nearest even (a wrong reading, for the teeth check)."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_weight_rounding_matches_hand_derived_float16():
    # tests/golden/beam_weight_rounding.txt: parts rounded separately to
    # binary16, nearest with ties to even, overflow to infinity
    w, re, im = _rounding_cases()
    with np.errstate(over="ignore"):
        got = beam.round_weights(w)
    np.testing.assert_array_equal(got.real, re)
    np.testing.assert_array_equal(got.imag, im)


def test_weight_rounding_pins_reject_other_readings():
    # each plausible misreading disagrees with at least one hand-derived row
    w, re, im = _rounding_cases()
    want = re + 1j * im
    fin = np.isfinite(re)

    def differs(r):
        return bool(np.any(r[fin] != want[fin]))

    assert differs(_rtz16(w.real) + 1j * _rtz16(w.imag))            # toward zero
    assert differs(_bf16(w.real) + 1j * _bf16(w.imag))              # bfloat16
    mag = np.abs(w)
    with np.errstate(over="ignore", invalid="ignore"):
        m16 = mag.astype(np.float16).astype(np.float64)
        by_mag = np.where(mag > 0, w * (m16 / np.where(mag > 0, mag, 1)), 0)
    assert differs(by_mag)                                           # magnitude rounded, angle kept
    with np.errstate(over="ignore"):
        assert differs(w.real.astype(np.float32).astype(np.float64) + 1j * w.imag)  # float32 only
