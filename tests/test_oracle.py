"""The CPU oracle against its pins (no GPU).

Also shows the pins have teeth: textual mutations of the oracle's C source
(a flipped sign, a dropped term, swapped nibbles, a wrong triangle index, a
wrong negative decode) are compiled into throw-away libraries and each must
fail at least one pin.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth
from tests import pins


def test_decode_golden():
    for b, re, im in pins.read_decode_golden():
        assert oracle.decode(b) == (re, im), hex(b)


def test_decode_exhaustive():
    table = pins.encoder_decode_table()
    for b in range(256):
        assert oracle.decode(b) == table[b] == pins.sign_extend_decode(b)


def test_unpack_matches_table():
    x = np.arange(256, dtype=np.uint8).reshape(4, 64)
    u = oracle.unpack(x)
    table = pins.encoder_decode_table()
    for b in range(256):
        assert tuple(u.reshape(256, 2)[b]) == table[b]


def test_hand_example():
    pins.pin_hand_example(oracle.correlate)


def test_single_product_all_pairs():
    pins.pin_single_product_all_pairs(oracle.correlate)


def test_autocorrelations():
    pins.pin_autocorrelations(oracle.correlate, synth.uniform_bytes((64, 3, 10), 3))


def test_hermitian():
    pins.pin_hermitian(oracle.correlate, synth.uniform_bytes((40, 2, 13), 4))


def test_rank1_closed_form():
    pins.pin_rank1(oracle.correlate)


def test_invariants():
    pins.pin_invariants(oracle.correlate, synth.uniform_bytes((57, 3, 11), 8))


def test_multiply_by_i():
    pins.pin_multiply_by_i(oracle.correlate)


def test_bound_arithmetic():
    pins.pin_bound(oracle.correlate)


def test_brute_force():
    pins.pin_brute_force(oracle.correlate)


def test_thread_count_independent():
    x = synth.uniform_bytes((33, 7, 9), 9)
    ref = oracle.correlate(x, nthreads=1)
    for n in (2, 3, 8, 64):
        np.testing.assert_array_equal(oracle.correlate(x, nthreads=n), ref)


def test_correlate_one_matches_full():
    x = synth.uniform_bytes((50, 3, 8), 10)
    v = oracle.correlate(x)
    for c in range(3):
        for i in range(8):
            for j in range(i + 1):
                assert oracle.correlate_one(x, c, i, j) == tuple(v[c, oracle.tri_index(i, j)])


def test_empty_inputs():
    assert oracle.correlate(np.zeros((0, 2, 3), np.uint8)).shape == (2, 6, 2)
    assert (oracle.correlate(np.zeros((0, 2, 3), np.uint8)) == 0).all()
    assert oracle.correlate(np.zeros((5, 0, 3), np.uint8)).shape == (0, 6, 2)
    assert oracle.correlate(np.zeros((5, 2, 0), np.uint8)).shape == (2, 0, 2)


def test_tone_channel_statistics():
    """Generator sanity: in the tone channel the mean cross power is close to
    the tone power 3^2 = 9 with zero relative phase (config 'tiny' has
    phi_i = 0); elsewhere it is close to 0."""
    x = synth.config_voltages("tiny")
    v = oracle.correlate(x).astype(np.float64) / x.shape[0]
    N = x.shape[2]
    cross = np.array([oracle.tri_index(i, j) for i in range(N) for j in range(i)])
    tone = v[10, cross, 0].mean()
    other = np.delete(v[:, cross, 0], 10, axis=0).mean()
    assert 8.0 < tone < 9.8, tone
    assert abs(other) < 0.3, other
    assert abs(v[10, cross, 1].mean()) < 0.5


def test_generator_reproducible_and_thread_independent():
    a = synth.voltages(8, 4, 300, seed=5, threads=1, random_phase=True)
    b = synth.voltages(8, 4, 300, seed=5, threads=4, random_phase=True)
    c = synth.voltages(8, 4, 300, seed=6, threads=4, random_phase=True)
    np.testing.assert_array_equal(a, b)
    assert (a != c).any()
    z = pins.complex_samples(a)
    assert z.real.min() >= -8 and z.real.max() <= 7


# ---------------------------------------------------------------------------
# mutation tests: every plausible mistake must fail some pin
# ---------------------------------------------------------------------------

MUTANTS = {
    "conj_on_wrong_side": ("im += (int64_t)bi * aj - (int64_t)ai * bj;",
                           "im += (int64_t)ai * bj - (int64_t)bi * aj;"),
    "dropped_imag_imag_term": ("re += (int64_t)ai * aj + (int64_t)bi * bj;",
                               "re += (int64_t)ai * aj;"),
    "nibbles_swapped": ("*re = oracle_nibble_value((unsigned)b >> 4);\n    *im = oracle_nibble_value((unsigned)b);",
                        "*im = oracle_nibble_value((unsigned)b >> 4);\n    *re = oracle_nibble_value((unsigned)b);"),
    "unsigned_nibbles": ("return (nib < 8u) ? (int)nib : (int)nib - 16;",
                         "return (int)nib;"),
    "minus_eight_as_plus_eight": ("return (nib < 8u) ? (int)nib : (int)nib - 16;",
                                  "return (nib <= 8u) ? (int)nib : (int)nib - 16;"),
    "wrong_triangle_index": (": i * (i + 1) / 2 + j;", ": j * (j + 1) / 2 + i - j;"),
    "channel_stride_wrong": ("job->x[(t * C + c) * N + j]", "job->x[(t * C) * N + j]"),
}


def _build_mutant(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "xcorr_oracle.c")).read()
    old, new = MUTANTS[name]
    assert old in src, f"mutation anchor for {name} not found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-pthread", "-o",
                           str(so), str(path)])
    lib = ctypes.CDLL(str(so))
    i64, p = ctypes.c_int64, ctypes.c_void_p
    lib.oracle_correlate.argtypes = [p, i64, i64, i64, p, ctypes.c_int, ctypes.c_int]

    def correlate(x, full_square=False):
        x = np.ascontiguousarray(x, dtype=np.uint8)
        T, C, N = x.shape
        nbl = N * N if full_square else N * (N + 1) // 2
        out = np.zeros((C, nbl, 2), dtype=np.int64)
        lib.oracle_correlate(x.ctypes.data, T, C, N, out.ctypes.data,
                             int(full_square), 4)
        return out.reshape(C, N, N, 2) if full_square else out
    return correlate


def _pin_suite(correlate):
    x = synth.uniform_bytes((21, 3, 7), 12)
    yield lambda: pins.pin_hand_example(correlate)
    yield lambda: pins.pin_single_product_all_pairs(correlate)
    yield lambda: pins.pin_autocorrelations(correlate, x)
    yield lambda: pins.pin_hermitian(correlate, x)
    yield lambda: pins.pin_rank1(correlate)
    yield lambda: pins.pin_brute_force(correlate)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    correlate = _build_mutant(name, tmp_path)
    failed = 0
    for pin in _pin_suite(correlate):
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed > 0, f"mutant {name} passed every pin"
