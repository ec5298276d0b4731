"""GPU beamformer vs the float64 oracle (same float16-rounded weights).

The kernel accumulates float32 products of biased voltages u = v + 8 and
float16 weights, then removes the bias 8 sum_k W'[n][k] (W' the real
operand: Re w / -Im w for a beam's real part, Im w / Re w for its imaginary
part).  Each product is exact in float32; an accumulation over K = 2 Npad
terms in any order errs by at most (K + 8) u (15 sum|W'| + 8 |sum W'|) with
u = 2^-24, and the final FFMA adds u |y|.  That bound is checked per output,
and the normwise relative error must stay below 1e-4."""
import numpy as np
import pytest

import synth
from oracle import beam as obeam

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


@pytest.fixture(scope="module")
def bm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_00720_b300 import beam
    return beam


def bound(w, npad, y):
    wr = obeam.round_weights(w)                       # [C][B][N]
    s_abs = np.abs(wr.real).sum(-1) + np.abs(wr.imag).sum(-1)
    s_re = np.abs((wr.real - wr.imag).sum(-1))
    s_im = np.abs((wr.imag + wr.real).sum(-1))
    k = 2 * npad + 8
    b_re = k * U * (15 * s_abs + 8 * s_re)
    b_im = k * U * (15 * s_abs + 8 * s_im)
    return b_re[None] + 2 * U * np.abs(y.real), b_im[None] + 2 * U * np.abs(y.imag)


def run(bm, x, w, B):
    import torch
    T, C, N = x.shape
    f = bm.Beamformer(N, C, B, max(T, 1))
    f.set_weights(torch.from_numpy(np.ascontiguousarray(w)).cuda())
    y = f.form(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    f.check()
    out = y.cpu().numpy()
    f.close()
    return out


def check(got, x, w):
    ref = obeam.beamform(x, w)
    npad = -(-x.shape[2] // 64) * 64
    br, bi = bound(w, npad, ref)
    er, ei = np.abs(got.real - ref.real), np.abs(got.imag - ref.imag)
    assert np.all(er <= br) and np.all(ei <= bi), (er.max(), ei.max())
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref) + 1e-30


SHAPES = [  # (N, C, B, T): input padding, time tails, every beam count, multi-stage
    (64, 2, 8, 128),
    (128, 3, 16, 200),
    (96, 2, 16, 300),
    (528, 2, 8, 257),
    (64, 1, 64, 128),
    (256, 4, 32, 512),
    (512, 4, 16, 1000),
    (16, 1, 24, 1),
    (1024, 2, 16, 256),   # weights too large to stay resident: streamed per group of stages
    (256, 40, 16, 128),   # many channels per CTA: resident weights reloaded at channel changes
    (400, 3, 16, 200),    # time along N: a partial last 128-input stage (zero-filled inputs)
    (512, 2, 16, 1),      # time along N: one sample per channel
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_beamformer_matches_oracle(bm, shape):
    N, C, B, T = shape
    x = synth.voltages(N, C, T, seed=N + C + B, random_phase=True, tone_chan=0)
    w = synth.beam_weights(N, C, B, seed=B + N)
    check(run(bm, x, w, B), x, w)


def test_random_weights_and_uniform_bytes(bm):
    N, C, B, T = 192, 3, 16, 384
    rng = np.random.default_rng(5)
    x = synth.uniform_bytes((T, C, N), seed=6)
    w = (rng.standard_normal((C, B, N)) + 1j * rng.standard_normal((C, B, N))).astype(np.complex64)
    check(run(bm, x, w, B), x, w)


def test_weight_dynamic_range(bm):
    """Weights of one channel spanning 2^-20 .. 1 in magnitude (below 2^-18 of
    the largest the time-along-N kernel's e4m3 terms are no longer exact, and
    err by less than 2^-28 of it), a channel of zero weights and one of large
    weights (~1e4); 8 beams, so half of that kernel's operand rows are zero."""
    N, C, B, T = 256, 3, 8, 384
    rng = np.random.default_rng(12)
    mag = 2.0 ** rng.uniform(-20, 0, (C, B, N))
    w = (mag * np.exp(2j * np.pi * rng.random((C, B, N)))).astype(np.complex64)
    w[1] = 0
    w[2] *= np.float32(1.0e4)
    x = synth.voltages(N, C, T, seed=12, random_phase=True)
    got = run(bm, x, w, B)
    assert np.all(got[:, 1] == 0)
    check(got, x, w)


def test_extreme_samples(bm):
    N, C, B, T = 128, 2, 8, 256
    x = np.full((T, C, N), 0x88, np.uint8)            # -8 - 8i everywhere
    w = synth.beam_weights(N, C, B, seed=3) * N        # unit-magnitude phases
    check(run(bm, x, w, B), x, w)


def test_steered_tone_on_gpu(bm):
    rng = np.random.default_rng(9)
    T, N = 256, 64
    s = rng.integers(-7, 8, T)
    k = rng.integers(0, 4, N)
    u = np.array([1, 1j, -1, -1j])[k]
    xs = s[:, None] * u[None, :]
    x = synth.pack(xs.real.astype(int), xs.imag.astype(int))[:, None, :].copy()
    x = np.repeat(x, 2, axis=1)                        # C = 2
    w = np.zeros((2, 8, N), np.complex64)
    w[:, 0, :] = np.conj(u)
    got = run(bm, x, w, 8)
    np.testing.assert_allclose(got[:, 0, 0], N * s, rtol=0, atol=1e-3)


def test_argument_errors(bm):
    import torch
    from paper_1708_00720_b300 import xengine as xe
    with pytest.raises(xe.XEngineError):
        bm.Beamformer(64, 1, 12, 128)                  # beams not a multiple of 8
    with pytest.raises(xe.XEngineError) as e:
        bm.Beamformer(20, 1, 8, 128)                   # N not a multiple of 16
    assert e.value.status == xe.XE_ERR_ALIGNMENT
    f = bm.Beamformer(64, 1, 8, 128)
    x = torch.zeros((128, 1, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(xe.XEngineError):
        f.form(x)                                      # weights not set
    f.set_weights(torch.zeros((1, 8, 64), dtype=torch.complex64, device="cuda"))
    with pytest.raises(xe.XEngineError):
        f.form(torch.zeros((129, 1, 64), dtype=torch.uint8, device="cuda"))   # above max_ntime
    assert f.form(x[:0]).shape == (0, 1, 8)
    f.close()


def test_full_size_sampled(bm):
    """512 inputs, 256 channels, 8192 samples, 16 beams; outputs checked one by one."""
    import torch
    p = synth.BEAM_CONFIG
    N, C, T, B = p["ninput"], p["nchan"], p["ntime"], p["nbeam"]
    x = synth.voltages(N, C, T, seed=p["seed"], random_phase=True)
    w = synth.beam_weights(N, C, B, seed=p["seed"])
    y = run(bm, x, w, B)
    rng = np.random.default_rng(1)
    npad = 512
    br, bi = bound(w, npad, np.zeros((1, C, B), complex))
    for _ in range(300):
        t, c, b = int(rng.integers(T)), int(rng.integers(C)), int(rng.integers(B))
        e = obeam.beamform_one(x, w, t, c, b)
        assert abs(y[t, c, b].real - e.real) <= br[0, c, b] + 2 * U * abs(e.real)
        assert abs(y[t, c, b].imag - e.imag) <= bi[0, c, b] + 2 * U * abs(e.imag)
    for t in (0, T - 1):
        np.testing.assert_allclose(y[t], obeam.beamform(x[t:t + 1], w)[0], rtol=1e-3, atol=1e-4)
