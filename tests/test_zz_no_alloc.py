"""The allocation-free entry point (xe_correlate_noalloc) against the plan
entry points, through the C ABI.

Callers that cannot allocate device memory (a framework that owns all device
memory, or a real-time pipeline that must not allocate while observing) use
xe_correlate_noalloc, whose scratch is a fixed array inside the library.  Its
output must equal that of xe_correlate + xe_integrate on the same gulp, and
it must stay equal on consecutive calls, since every call reuses the same
scratch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_00720_b300 import xengine
    fn = xengine.library().xe_correlate_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    chk = xengine.library().xe_correlate_noalloc_check
    chk.argtypes = [ctypes.c_void_p]
    chk.restype = ctypes.c_int
    return xengine


def check(xe):
    import torch
    return xe.library().xe_correlate_noalloc_check(torch.cuda.current_stream().cuda_stream)


def noalloc(xe, gulp, out, out_type):
    import torch
    T, C, N = gulp.shape
    return xe.library().xe_correlate_noalloc(gulp.data_ptr(), T, C, N, out_type, out.data_ptr(),
                                             torch.cuda.current_stream().cuda_stream)


def plan_result(xe, gulp, out):
    T, C, N = gulp.shape
    eng = xe.XEngine(N, C, max(T, 1), "fp8", out)
    eng.correlate(gulp)
    v = eng.integrate()
    eng.check()
    eng.close()
    return v


@pytest.mark.parametrize("out", ["ci32", "cf32"])
def test_noalloc_matches_plan_two_calls_in_a_row(xe, out):
    import torch
    out_type = xe.XE_OUT_CF32 if out == "cf32" else xe.XE_OUT_CI32
    dtype = torch.float32 if out == "cf32" else torch.int32
    for seed, (N, C, T) in ((31, (272, 9, 1000)), (32, (144, 20, 333))):
        g = torch.from_numpy(synth.voltages(N, C, T, seed=seed, random_phase=True)).cuda()
        want = plan_result(xe, g, out)
        got = torch.full((C, N * (N + 1) // 2, 2), -7, dtype=dtype, device="cuda")
        assert noalloc(xe, g, got, out_type) == xe.XE_OK
        assert check(xe) == xe.XE_OK
        np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy())


def test_noalloc_repeated_call_same_input(xe):
    import torch
    g = torch.from_numpy(synth.voltages(512, 8, 2048, seed=33, random_phase=True)).cuda()
    want = plan_result(xe, g, "ci32").cpu().numpy()
    for _ in range(2):
        got = torch.zeros((8, 512 * 513 // 2, 2), dtype=torch.int32, device="cuda")
        assert noalloc(xe, g, got, xe.XE_OUT_CI32) == xe.XE_OK
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), want)


def test_noalloc_rejects_sizes_beyond_its_scratch(xe):
    import torch
    g = torch.zeros((32, 64, 512), dtype=torch.uint8, device="cuda")  # 64 x 131328 > 2^21
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    assert noalloc(xe, g, out, xe.XE_OUT_CI32) == xe.XE_ERR_SHAPE


def test_noalloc_long_gulp_runs_several_launches(xe):
    # 40000 samples exceed one launch's exact-float32 bound (32768), so the
    # call runs two launches, the second adding into the shared scratch;
    # checked against the CPU oracle, twice in a row
    import torch
    import oracle
    N, C, T = 128, 16, 40000
    x = synth.voltages(N, C, T, seed=34, random_phase=True)
    want = oracle.correlate(x)
    g = torch.from_numpy(x).cuda()
    for _ in range(2):
        got = torch.full((C, N * (N + 1) // 2, 2), 5, dtype=torch.int32, device="cuda")
        assert noalloc(xe, g, got, xe.XE_OUT_CI32) == xe.XE_OK
        assert check(xe) == xe.XE_OK
        np.testing.assert_array_equal(got.cpu().numpy().astype(np.int64), want)


def test_noalloc_zero_samples_writes_zeros(xe):
    import torch
    N, C = 144, 3
    g = torch.zeros((1, C, N), dtype=torch.uint8, device="cuda")
    for out_type, dtype in ((xe.XE_OUT_CI32, torch.int32), (xe.XE_OUT_CF32, torch.float32)):
        got = torch.full((C, N * (N + 1) // 2, 2), 9, dtype=dtype, device="cuda")
        assert xe.library().xe_correlate_noalloc(g.data_ptr(), 0, C, N, out_type, got.data_ptr(),
                                                 torch.cuda.current_stream().cuda_stream) == xe.XE_OK
        assert check(xe) == xe.XE_OK
        assert int(torch.count_nonzero(got)) == 0
