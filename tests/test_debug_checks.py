"""The index-checked debug build (libxengine_debug.so, XE_DEBUG_CHECKS)
through the C ABI: every global store of the X-engine kernels is checked
against its buffer, an access outside it is skipped and reported by
xe_plan_check as XE_ERR_DEVICE_INDEX.  This stands in for a device memory
checker: shapes that exercise every write path (ragged tiles, transposed
odd-one-out tiles, time-sliced leftover units with their combine kernel,
accumulation, long gulps split over launches) must come back bit-exact with
no index report."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SHAPES = [  # (N, C, T)
    (144, 2, 200),     # ragged tiles
    (272, 3, 129),     # odd tile count: transposed odd-one-out tiles
    (640, 12, 2048),   # 96 units on 74 clusters: 22 leftovers cut in two along time
    (128, 1, 40000),   # two launches, the second accumulating
]


@pytest.fixture(scope="module")
def dbg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_00720_b300 import xengine
    return xengine, xengine.debug_library()


def correlate(xe, lib, x, operand, out_type):
    import torch
    T, C, N = x.shape
    plan = ctypes.c_void_p()
    assert lib.xe_plan_create(ctypes.byref(plan), N, C, T, operand, out_type) == xe.XE_OK
    g = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    dt = torch.float32 if out_type == xe.XE_OUT_CF32 else torch.int32
    vis = torch.full((C, N * (N + 1) // 2, 2), 3, dtype=dt, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.xe_correlate(plan, g.data_ptr(), T, 0, s) == xe.XE_OK
    assert lib.xe_integrate(plan, vis.data_ptr(), s) == xe.XE_OK
    st = lib.xe_plan_check(plan)
    emit = torch.full_like(vis, 5)
    if out_type == xe.XE_OUT_CI32 and T <= 32768:
        assert lib.xe_correlate_emit(plan, g.data_ptr(), T, emit.data_ptr(), s) == xe.XE_OK
        st2 = lib.xe_plan_check(plan)
    else:
        st2 = xe.XE_OK
        emit = None
    lib.xe_plan_destroy(plan)
    return st, st2, vis.cpu().numpy().astype(np.int64), None if emit is None else emit.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("operand", ["fp8", "fp16", "int32"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"N{s[0]}C{s[1]}T{s[2]}")
def test_debug_build_reports_no_index_outside_a_buffer(dbg, shape, operand):
    xe, lib = dbg
    N, C, T = shape
    if operand == "int32" and T > 8192:
        pytest.skip("the int32 path's long-gulp case adds nothing here")
    x = synth.voltages(N, C, T, seed=N + C, random_phase=True)
    want = oracle.correlate(x)
    st, st2, got, emit = correlate(xe, lib, x, xe.OPERANDS[operand], xe.XE_OUT_CI32)
    assert st == xe.XE_OK, xe.xe_status_string(st)
    assert st2 == xe.XE_OK, xe.xe_status_string(st2)
    np.testing.assert_array_equal(got, want)
    if emit is not None:
        np.testing.assert_array_equal(emit, want)
