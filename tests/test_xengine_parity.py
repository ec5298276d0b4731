"""GPU X-engine vs the CPU oracle, element by element (bit-exact).

Every operand path (tcgen05 e4m3, tcgen05 f16, CUDA-core int32) is called
through the C ABI on the same seeded bytes the oracle reads.  Small cases
are compared in full; the full-size workloads are compared on sampled
baselines computed one by one by the oracle, plus properties that hold at
any size.
"""
import functools

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

OPS = ["fp8", "fp16", "int32"]


@pytest.fixture(scope="module")
def xe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_00720_b300 import xengine
    return xengine


def run(xe, x, operand, out="ci32", max_ntime=None, emit=False):
    """Visibilities of one gulp through correlate + integrate, or (emit) through
    the fused one-gulp call the benchmark step times."""
    import torch
    T, C, N = x.shape
    eng = xe.XEngine(N, C, max_ntime or max(T, 1), operand, out)
    g = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    if emit:
        v = eng.correlate_emit(g)
    else:
        eng.correlate(g)
        v = eng.integrate()
    torch.cuda.synchronize()
    eng.check()
    assert eng.samples() == (0 if emit else T)
    res = v.cpu().numpy()
    eng.close()
    if out == "cf32":
        assert np.all(res == np.round(res))
    return res.astype(np.int64)


SMALL_SHAPES = [  # (N, C, T): tile-ragged inputs, time tails, single samples
    (16, 64, 1024),   # the tiny workload's shape
    (48, 3, 100),
    (144, 2, 33),
    (272, 2, 257),
    (128, 1, 1),
    (256, 5, 64),
    (16, 1, 31),
    (400, 1, 96),
    # 128-input tiles per side nt = 5, 6, 7: the tensor-core paths group tile
    # pairs by J column two at a time, compute a column's odd one out as its
    # transpose and, for an odd total (nt = 5, 6), repeat one tile unwritten
    (640, 1, 40),
    (736, 2, 33),
    (896, 1, 64),
    # a unit's first stages are issued in two halves (real parts while the
    # epilogue still reads D_im); stage counts at and just past the
    # four-stage operand ring (e4m3 stages are 128 samples, f16 64)
    (144, 3, 512),
    (272, 2, 640),
    (144, 2, 256),
]


@pytest.mark.parametrize("operand", OPS)
@pytest.mark.parametrize("shape", SMALL_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_small_full_parity(xe, operand, shape):
    N, C, T = shape
    x = synth.voltages(N, C, T, seed=N * 7 + C + T, random_phase=True)
    np.testing.assert_array_equal(run(xe, x, operand), oracle.correlate(x))


@pytest.mark.parametrize("operand", OPS)
def test_tiny_workload(xe, operand):
    x = synth.config_voltages("tiny")
    np.testing.assert_array_equal(run(xe, x, operand), oracle.correlate(x))


@pytest.mark.parametrize("operand", OPS)
def test_uniform_bytes_every_nibble(xe, operand):
    x = synth.uniform_bytes((300, 3, 160), seed=21)
    np.testing.assert_array_equal(run(xe, x, operand), oracle.correlate(x))


@pytest.mark.parametrize("operand", OPS)
def test_extreme_values_long_gulp(xe, operand):
    """Samples drawn from the corners of the 4-bit square over 32768 samples:
    the largest float32 partial sums one tensor-core launch may hold."""
    rng = np.random.default_rng(5)
    corners = np.array([0x88, 0x77, 0x87, 0x78, 0x80, 0x08, 0x70, 0x07], dtype=np.uint8)
    x = corners[rng.integers(0, len(corners), (32768, 2, 128))]
    np.testing.assert_array_equal(run(xe, x, operand), oracle.correlate(x))


@pytest.mark.parametrize("operand", OPS)
def test_all_minus_eight(xe, operand):
    x = np.full((32768, 1, 16), 0x88, dtype=np.uint8)
    v = run(xe, x, operand)
    assert (v[..., 0] == 128 * 32768).all() and (v[..., 1] == 0).all()


@pytest.mark.parametrize("operand", ["fp8", "fp16"])
def test_gulp_longer_than_one_launch(xe, operand):
    x = synth.voltages(32, 2, 40000, seed=3)
    np.testing.assert_array_equal(run(xe, x, operand), oracle.correlate(x))


# Shapes whose pair units do not fill whole rounds of the 74 CTA pairs of a
# 148-SM B300: the units left over are cut along time over all pairs, each
# slice reduced with its own bias corrections and added with integer atomics
# (into a tile that the first slice to finish zeroes, when overwriting).
SPLIT_SHAPES = [  # (N, C, T)
    (16, 75, 4096),    # one unit per channel, one left over
    (16, 96, 4096),    # 22 left over, as at 512 inputs x 256 channels
    (144, 38, 2048),   # two units per channel; a leftover one repeats a tile unwritten
    (272, 25, 2048),   # three per channel; the leftover one holds a transposed tile
]


@functools.lru_cache(maxsize=None)
def _split_case(shape):
    N, C, T = shape
    x = synth.voltages(N, C, T, seed=N + 3 * C + T, random_phase=True)
    return x, oracle.correlate(x)


@pytest.mark.parametrize("operand", ["fp8", "fp16"])
@pytest.mark.parametrize("shape", SPLIT_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_time_sliced_leftover_units(xe, operand, shape):
    import torch
    N, C, T = shape
    x, ref = _split_case(shape)
    eng = xe.XEngine(N, C, T, operand)
    g = torch.from_numpy(x).cuda()
    for _ in range(2):   # the tiles' claim words must be back to zero for the second launch
        eng.correlate(g)
        v = eng.integrate().cpu().numpy()
        eng.check()
        np.testing.assert_array_equal(v, ref)
    eng.correlate(g, accumulate=True)
    v = eng.integrate().cpu().numpy()
    eng.check()
    np.testing.assert_array_equal(v, 2 * ref)
    eng.close()


@pytest.mark.parametrize("operand", OPS)
def test_correlate_emit(xe, operand):
    """A one-gulp integration written straight into the caller's buffer: the
    values of correlate + integrate, the buffer overwritten (not added to),
    the plan's own accumulator and sample count untouched."""
    import torch
    N, C, T = 272, 25, 2048      # leftover units cut along time on the tensor-core paths
    x, ref = _split_case((N, C, T))
    eng = xe.XEngine(N, C, T, operand)
    g = torch.from_numpy(x).cuda()
    eng.correlate(g[:100])
    before = eng.integrate().cpu().numpy()
    out = torch.full((C, eng.n_baselines, 2), 7, dtype=torch.int32, device="cuda")
    assert eng.correlate_emit(g, out) is out
    eng.check()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    np.testing.assert_array_equal(eng.integrate().cpu().numpy(), before)
    assert eng.samples() == 100
    eng.correlate_emit(g[:0], out)                   # an empty gulp: zero visibilities
    assert (out.cpu().numpy() == 0).all()
    eng.close()
    with pytest.raises(xe.XEngineError) as e:        # ci32 plans only
        f = xe.XEngine(N, C, T, operand, "cf32")
        try:
            f.correlate_emit(g, torch.empty((C, eng.n_baselines, 2), dtype=torch.int32, device="cuda"))
        finally:
            f.close()
    assert e.value.status == xe.XE_ERR_INVALID_ARG


@pytest.mark.parametrize("operand", ["fp8", "fp16"])
def test_correlate_emit_longer_than_one_launch(xe, operand):
    import torch
    x = synth.voltages(32, 2, 40000, seed=3)
    eng = xe.XEngine(32, 2, 40000, operand)
    out = eng.correlate_emit(torch.from_numpy(x).cuda())
    eng.check()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.correlate(x))
    eng.close()


@pytest.mark.parametrize("operand", OPS)
def test_accumulate_and_reset(xe, operand):
    import torch
    x = synth.voltages(144, 3, 500, seed=9, random_phase=True)
    eng = xe.XEngine(144, 3, 300, operand)
    g1 = torch.from_numpy(x[:300].copy()).cuda()
    g2 = torch.from_numpy(x[300:].copy()).cuda()
    eng.correlate(g1)
    eng.correlate(g2, accumulate=True)
    assert eng.samples() == 500
    v = eng.integrate().cpu().numpy()
    eng.check()
    np.testing.assert_array_equal(v, oracle.correlate(x))
    eng.correlate(g2)  # overwrite
    np.testing.assert_array_equal(eng.integrate().cpu().numpy(), oracle.correlate(x[300:]))
    eng.reset()
    assert eng.samples() == 0
    assert (eng.integrate().cpu().numpy() == 0).all()
    eng.correlate(g1[:0], accumulate=True)  # empty gulp adds nothing
    assert (eng.integrate().cpu().numpy() == 0).all()
    eng.close()


@pytest.mark.parametrize("operand", OPS)
def test_cf32_output(xe, operand):
    x = synth.voltages(64, 4, 200, seed=10)
    np.testing.assert_array_equal(run(xe, x, operand, out="cf32"), oracle.correlate(x))


def test_cf32_bound(xe):
    import torch
    T = xe.XE_MAX_SAMPLES_CF32
    eng = xe.XEngine(16, 1, T, "fp8", "cf32")
    g = torch.full((T, 1, 16), 0x88, dtype=torch.uint8, device="cuda")
    eng.correlate(g)  # exactly at the bound: 128 * T = 2^24
    v = eng.integrate().cpu().numpy()
    eng.check()
    assert (v[..., 0] == 2.0 ** 24).all() and (v[..., 1] == 0).all()
    with pytest.raises(xe.XEngineError) as e:
        eng.correlate(g[:1], accumulate=True)
    assert e.value.status == xe.XE_ERR_ACCUM_BOUND
    assert eng.samples() == T  # a rejected call changes nothing
    eng.close()


def test_ci32_bound(xe):
    import torch
    T = xe.XE_MAX_SAMPLES_CI32
    eng = xe.XEngine(16, 1, T, "fp8", "ci32")
    g = torch.full((T, 1, 16), 0x88, dtype=torch.uint8, device="cuda")
    eng.correlate(g)
    v = eng.integrate().cpu().numpy()
    eng.check()
    assert (v[..., 0] == 128 * T).all() and (v[..., 1] == 0).all()
    with pytest.raises(xe.XEngineError) as e:
        eng.correlate(g[:1], accumulate=True)
    assert e.value.status == xe.XE_ERR_ACCUM_BOUND
    eng.close()


def test_shape_and_alignment_errors(xe):
    import torch
    eng = xe.XEngine(32, 2, 64, "fp8")
    g = torch.zeros((65, 2, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(xe.XEngineError) as e:
        xe.xe_correlate(eng.plan, g, 65)
    assert e.value.status == xe.XE_ERR_SHAPE
    with pytest.raises(xe.XEngineError) as e:
        xe.xe_correlate(eng.plan, g.data_ptr() + 1, 8)
    assert e.value.status == xe.XE_ERR_ALIGNMENT
    vis = torch.zeros(2 * 528 * 2 + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(xe.XEngineError) as e:
        xe.xe_integrate(eng.plan, vis.data_ptr() + 4)
    assert e.value.status == xe.XE_ERR_ALIGNMENT
    eng.close()


def test_unpack(xe):
    import torch
    x = np.concatenate([np.arange(256, dtype=np.uint8),
                        synth.uniform_bytes(16 * 64 * 3 - 256, 3)]).reshape(3, 64, 16)
    eng = xe.XEngine(16, 64, 3, "fp8")
    g = torch.from_numpy(x).cuda()
    out = torch.empty((3, 64, 16, 2), dtype=torch.int8, device="cuda")
    xe.xe_unpack(eng.plan, g, out, 3)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.unpack(x))
    eng.close()


def test_host_end_to_end(xe):
    import torch
    x = synth.voltages(256, 8, 5000, seed=12, random_phase=True)
    eng = xe.XEngine(256, 8, 5000, "fp8")
    h_in = torch.from_numpy(x).pin_memory()
    h_out = eng.vis_empty(device="cpu", pin_memory=True)
    xe.xe_correlate_host(eng.plan, h_in, 5000, 0, h_out)
    eng.check()
    np.testing.assert_array_equal(h_out.numpy(), oracle.correlate(x))
    assert eng.samples() == 5000
    eng.close()


# ---------------------------------------------------------------- full size
def sampled_check(v, x, rng, nsamp=1500):
    T, C, N = x.shape
    cs = rng.integers(0, C, nsamp)
    ii = rng.integers(0, N, nsamp)
    jj = (rng.random(nsamp) * (ii + 1)).astype(np.int64)
    # always include the tile corners and the last input
    extra = [(0, 0), (N - 1, 0), (N - 1, N - 1), (127, 127), (128, 127), (min(N - 1, 255), 128)]
    for (i, j) in extra:
        cs = np.append(cs, rng.integers(0, C))
        ii = np.append(ii, i)
        jj = np.append(jj, j)
    for c, i, j in zip(cs, ii, jj):
        want = oracle.correlate_one(x, int(c), int(i), int(j))
        got = tuple(v[c, oracle.tri_index(int(i), int(j))])
        assert got == want, (c, i, j, got, want)


def properties_check(v, x):
    T, C, N = x.shape
    diag = np.array([oracle.tri_index(i, i) for i in range(N)])
    assert (v[:, diag, 1] == 0).all()
    assert (v[:, diag, 0] >= 0).all()
    assert np.abs(v[..., 0]).max() <= 128 * T


@pytest.mark.parametrize("operand", ["fp8", "int32"])
def test_lwa_workload_sampled(xe, operand):
    """512 inputs, 256 channels, 8192 samples in the benchmark's launch
    configuration (the fused one-gulp call), equal to correlate + integrate."""
    x = synth.config_voltages("lwa")
    v = run(xe, x, operand, emit=True)
    np.testing.assert_array_equal(v, run(xe, x, operand))
    properties_check(v, x)
    sampled_check(v, x, np.random.default_rng(1))
    # autocorrelations of a few channels in full
    for c in (0, 10, 255):
        for i in range(0, 512, 37):
            assert tuple(v[c, oracle.tri_index(i, i)]) == oracle.correlate_one(x, c, i, i)


@pytest.mark.parametrize("operand", ["fp8", "fp16"])
def test_large_n_workload_sampled(xe, operand):
    x = synth.config_voltages("large_n")
    v = run(xe, x, operand, emit=True)
    np.testing.assert_array_equal(v, run(xe, x, operand))
    properties_check(v, x)
    sampled_check(v, x, np.random.default_rng(2))


@pytest.mark.parametrize("operand", OPS)
def test_maximum_inputs_sampled(xe, operand):
    """8192 inputs (the largest accepted), one channel, a ragged 200-sample
    gulp: sampled baselines one by one against the oracle, plus the
    properties that hold at any size."""
    x = synth.uniform_bytes((200, 1, 8192), seed=12)
    v = run(xe, x, operand)
    properties_check(v, x)
    sampled_check(v, x, np.random.default_rng(3))
    for i, j in ((8191, 0), (8191, 8191), (4096, 4095), (128, 127), (8191, 8064)):
        assert tuple(v[0, oracle.tri_index(i, j)]) == oracle.correlate_one(x, 0, i, j)


# ----------------------------------------------------- batched launches
def test_batched_launch_of_several_problems(xe):
    """Four problems of different array sizes (ragged tiles, a transposed odd
    tile, more units than clusters) in ONE launch, one of them accumulating
    onto an earlier gulp: each plan's visibilities equal the oracle's."""
    import torch
    shapes = [(512, 8, 1024), (272, 5, 333), (144, 3, 2048), (1024, 2, 256)]
    engs, xs, gs = [], [], []
    for k, (N, C, T) in enumerate(shapes):
        engs.append(xe.XEngine(N, C, 2 * T, "fp8"))
        xs.append(synth.voltages(N, C, T, seed=90 + k, random_phase=True))
        gs.append(torch.from_numpy(xs[-1]).cuda())
    # plan 2 already holds an earlier gulp; the batch adds to it
    x_prev = synth.voltages(144, 3, 700, seed=99, random_phase=True)
    engs[2].correlate(torch.from_numpy(x_prev).cuda())
    launches0 = [xe.xe_plan_launch_count(e.plan) for e in engs]
    acc = [0, 0, 1, 0]
    xe.xe_correlate_batch([e.plan for e in engs], gs, [g.shape[0] for g in gs], acc)
    torch.cuda.synchronize()
    for k, e in enumerate(engs):
        e.check()
        assert xe.xe_plan_launch_count(e.plan) == launches0[k] + 1
        got = e.integrate().cpu().numpy().astype(np.int64)
        want = oracle.correlate(xs[k])
        if acc[k]:
            want = want + oracle.correlate(x_prev)
            assert e.samples() == 700 + shapes[k][2]
        np.testing.assert_array_equal(got, want)
        e.close()


def test_batched_launch_matches_single_launches_at_lwa_scale(xe):
    """Two 512-input problems of 64 channels each (the shapes the serving
    workload batches): one batched launch equals two plan calls."""
    import torch
    x1 = synth.voltages(512, 64, 1024, seed=95, random_phase=True)
    x2 = synth.voltages(256, 64, 1024, seed=96, random_phase=True)
    e1, e2 = xe.XEngine(512, 64, 1024, "fp8"), xe.XEngine(256, 64, 1024, "fp8")
    g1, g2 = torch.from_numpy(x1).cuda(), torch.from_numpy(x2).cuda()
    xe.xe_correlate_batch([e1.plan, e2.plan], [g1, g2], [1024, 1024], [0, 0])
    v1, v2 = e1.integrate().cpu().numpy(), e2.integrate().cpu().numpy()
    e1.check(); e2.check()
    np.testing.assert_array_equal(v1, run(xe, x1, "fp8"))
    np.testing.assert_array_equal(v2, run(xe, x2, "fp8"))
    sampled_check(v1.astype(np.int64), x1, np.random.default_rng(4), nsamp=300)
    e1.close(); e2.close()


def test_batched_launch_argument_errors(xe):
    import ctypes
    import torch
    lib = xe.library()
    e8 = xe.XEngine(128, 2, 40000, "fp8")
    e16 = xe.XEngine(128, 2, 64, "fp16")
    g = torch.zeros((40000, 2, 128), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream

    def call(plans, T, acc=0):
        n = len(plans)
        P = (ctypes.c_void_p * max(n, 1))(*plans)
        G = (ctypes.c_void_p * max(n, 1))(*([g.data_ptr()] * n))
        Ts = (ctypes.c_int * max(n, 1))(*([T] * n))
        A = (ctypes.c_int * max(n, 1))(*([acc] * n))
        return lib.xe_correlate_batch(n, P, G, Ts, A, s)

    assert call([], 64) == xe.XE_ERR_INVALID_ARG
    assert call([e8.plan] * 9, 64) == xe.XE_ERR_INVALID_ARG
    assert call([e8.plan, e8.plan], 64) == xe.XE_ERR_INVALID_ARG          # one plan twice
    assert call([e8.plan, e16.plan], 64) == xe.XE_ERR_INVALID_ARG         # not e4m3
    assert call([e8.plan], 40000) == xe.XE_ERR_SHAPE                      # more than one launch
    assert call([e8.plan], 64, acc=2) == xe.XE_ERR_INVALID_ARG
    assert xe.xe_plan_launch_count(e8.plan) == 0
    e8.close(); e16.close()


def test_dp4a_probe_rate(xe):
    """The int32 path's ceiling: on B300 dp4a issues to the FMA-heavy pipe
    only, one warp instruction every other clock per scheduler, i.e. 64 dp4a
    per SM per clock.  The probe runs one CTA per SM, so each CTA's clock
    span is its SM's; a reading near 128 would mean CTAs shared an SM."""
    rate = xe.dp4a_rate_per_sm_clock()
    assert 56.0 <= rate <= 66.0, rate
