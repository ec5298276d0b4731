"""Pins for the X-engine oracle: facts fixed by the paper and by mathematics.

Each pin takes a ``correlate(x, full_square=False) -> int64 array`` callable
(the oracle's signature) so the same pins can be run against deliberately
broken copies of the oracle to show that every plausible mistake fails at
least one of them.  Nothing here re-types the oracle's formulas: values come
from an encoder-inverted decode table, Python complex-integer arithmetic,
closed forms and an independent numpy einsum.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def encoder_decode_table() -> dict[int, tuple[int, int]]:
    """byte -> (re, im), built by ENCODING every pair and inverting the map.

    Encoding is Python's own two's-complement masking of negative ints, the
    opposite direction of the oracle's decoder.
    """
    table = {}
    for re in range(-8, 8):
        for im in range(-8, 8):
            b = ((re & 0xF) << 4) | (im & 0xF)
            assert b not in table
            table[b] = (re, im)
    assert len(table) == 256
    return table


def sign_extend_decode(b: int) -> tuple[int, int]:
    """Second independent decode: place each nibble in the top of a signed
    byte and let int.from_bytes sign-extend it."""
    hi = int.from_bytes(bytes([b & 0xF0]), "big", signed=True) // 16
    lo = int.from_bytes(bytes([(b & 0x0F) << 4]), "big", signed=True) // 16
    return hi, lo


def complex_samples(x: np.ndarray) -> np.ndarray:
    """uint8 array -> complex128 array via the encoder-inverted table."""
    t = encoder_decode_table()
    lut = np.array([complex(*t[b]) for b in range(256)])
    return lut[x]


def read_decode_golden() -> list[tuple[int, int, int]]:
    rows = []
    with open(os.path.join(GOLDEN, "decode_examples.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                b, re, im = line.split()
                rows.append((int(b, 16), int(re), int(im)))
    return rows


def read_hand_example():
    with open(os.path.join(GOLDEN, "hand_example.txt")) as f:
        lines = [l.strip() for l in f if l.strip() and not l.startswith("#")]
    head = dict(kv.split("=") for kv in lines[0].split()[1:4])
    data = bytes.fromhex("".join(lines[0].split("bytes=")[1].split()))
    T, C, N = int(head["T"]), int(head["C"]), int(head["N"])
    x = np.frombuffer(data, dtype=np.uint8).reshape(T, C, N)
    out = np.array([int(v) for v in lines[1].split()[1:]], dtype=np.int64)
    return x, out.reshape(C, N * (N + 1) // 2, 2)


def einsum_reference(x: np.ndarray) -> np.ndarray:
    """Independent exact path: numpy int64 einsums over decoded parts."""
    z = complex_samples(x)
    a = z.real.astype(np.int64)
    b = z.imag.astype(np.int64)
    re = np.einsum("tci,tcj->cij", a, a) + np.einsum("tci,tcj->cij", b, b)
    im = np.einsum("tci,tcj->cij", b, a) - np.einsum("tci,tcj->cij", a, b)
    T, C, N = x.shape
    ii, jj = np.tril_indices(N)
    out = np.empty((C, len(ii), 2), dtype=np.int64)
    # np.tril_indices enumerates row-major (i ascending, j <= i ascending),
    # the same order as the packed index i(i+1)/2 + j.
    out[:, :, 0] = re[:, ii, jj]
    out[:, :, 1] = im[:, ii, jj]
    return out


def unpack_tri(v: np.ndarray, N: int) -> np.ndarray:
    """Packed [C][N(N+1)/2][2] -> complex [C][N][N] (lower triangle + mirror)."""
    C = v.shape[0]
    full = np.zeros((C, N, N), dtype=np.complex128)
    ii, jj = np.tril_indices(N)
    z = v[:, :, 0] + 1j * v[:, :, 1]
    full[:, ii, jj] = z
    full[:, jj, ii] = np.conj(z)
    return full


# --------------------------------------------------------------------------
# pins; each raises AssertionError on a mismatch
# --------------------------------------------------------------------------

def pin_hand_example(correlate):
    x, expect = read_hand_example()
    np.testing.assert_array_equal(correlate(x), expect)


def pin_single_product_all_pairs(correlate):
    """N=2, T=1: all 65536 byte pairs, one pair per channel."""
    b0, b1 = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    x = np.stack([b0.ravel(), b1.ravel()], axis=-1).astype(np.uint8)[None]
    v = correlate(x)
    z = complex_samples(x[0])
    z0, z1 = z[:, 0], z[:, 1]
    prod = z1 * np.conj(z0)  # exact: small complex integers in float64
    np.testing.assert_array_equal(v[:, 0, 0], (z0 * np.conj(z0)).real)
    np.testing.assert_array_equal(v[:, 0, 1], 0)
    np.testing.assert_array_equal(v[:, 1, 0], prod.real)
    np.testing.assert_array_equal(v[:, 1, 1], prod.imag)
    np.testing.assert_array_equal(v[:, 2, 0], (z1 * np.conj(z1)).real)
    np.testing.assert_array_equal(v[:, 2, 1], 0)


def pin_autocorrelations(correlate, x):
    v = correlate(x)
    N = x.shape[2]
    diag = np.array([i * (i + 1) // 2 + i for i in range(N)])
    z = complex_samples(x)
    np.testing.assert_array_equal(v[:, diag, 1], 0)
    assert (v[:, diag, 0] >= 0).all()
    power = (z * np.conj(z)).real.sum(axis=0)  # [C][N], exact small ints
    np.testing.assert_array_equal(v[:, diag, 0], power)


def pin_hermitian(correlate, x):
    """Full-square mode: V_ji = conj(V_ij); packed = its lower triangle."""
    full = correlate(x, full_square=True)
    np.testing.assert_array_equal(full[..., 0], np.swapaxes(full[..., 0], 1, 2))
    np.testing.assert_array_equal(full[..., 1], -np.swapaxes(full[..., 1], 1, 2))
    packed = correlate(x)
    N = x.shape[2]
    ii, jj = np.tril_indices(N)
    np.testing.assert_array_equal(packed, full[:, ii, jj, :])


def pin_rank1(correlate, T=300, N=12, C=2, seed=11):
    """x_t,i = s_t u_i with u_i in {1, i, -1, -i}: V_ij = u_i conj(u_j) sum|s|^2."""
    rng = np.random.default_rng(seed)
    s = (np.clip(np.rint(rng.normal(0, 3, (T, C))), -7, 7)
         + 1j * np.clip(np.rint(rng.normal(0, 3, (T, C))), -7, 7))
    u = np.array([1, 1j, -1, -1j])[rng.integers(0, 4, N)]
    z = s[:, :, None] * u[None, None, :]
    re = z.real.astype(np.int64)
    im = z.imag.astype(np.int64)
    x = (((re & 0xF) << 4) | (im & 0xF)).astype(np.uint8)
    v = correlate(x)
    power = (s * np.conj(s)).real.sum(axis=0)  # [C]
    expect = power[:, None, None] * (u[:, None] * np.conj(u)[None, :])[None]
    ii, jj = np.tril_indices(N)
    e = expect[:, ii, jj]
    np.testing.assert_array_equal(v[..., 0], e.real.astype(np.int64))
    np.testing.assert_array_equal(v[..., 1], e.imag.astype(np.int64))


def pin_invariants(correlate, x, seed=5):
    rng = np.random.default_rng(seed)
    T, C, N = x.shape
    v = correlate(x)
    # time permutation
    np.testing.assert_array_equal(correlate(x[rng.permutation(T)]), v)
    # splitting a gulp and integrating the parts
    if T >= 2:
        cut = T // 3 + 1
        np.testing.assert_array_equal(correlate(x[:cut]) + correlate(x[cut:]), v)
    # input permutation: V' = P V P^T
    perm = rng.permutation(N)
    vp = unpack_tri(correlate(x[:, :, perm]), N)
    vf = unpack_tri(v, N)
    np.testing.assert_array_equal(vp, vf[:, perm][:, :, perm])


def pin_multiply_by_i(correlate, T=200, C=2, N=9, seed=6):
    """Multiplying every input by i leaves V unchanged (no -8 imaginary part)."""
    rng = np.random.default_rng(seed)
    re = rng.integers(-8, 8, (T, C, N))
    im = rng.integers(-7, 8, (T, C, N))
    x = (((re & 0xF) << 4) | (im & 0xF)).astype(np.uint8)
    y = ((((-im) & 0xF) << 4) | (re & 0xF)).astype(np.uint8)  # i(a+ib) = -b+ia
    np.testing.assert_array_equal(correlate(y), correlate(x))


def pin_bound(correlate, T=131072):
    """All samples -8-8i: every visibility is 128 T (= 2^24 at T = 131072)."""
    x = np.full((T, 1, 2), 0x88, dtype=np.uint8)
    v = correlate(x)
    np.testing.assert_array_equal(v[..., 0], 128 * T)
    np.testing.assert_array_equal(v[..., 1], 0)


def pin_brute_force(correlate, seed=7):
    rng = np.random.default_rng(seed)
    for N in (1, 2, 3, 5, 17):
        for T in (1, 2, 3, 33):
            for C in (1, 3):
                x = rng.integers(0, 256, (T, C, N), dtype=np.uint8)
                np.testing.assert_array_equal(correlate(x), einsum_reference(x))
