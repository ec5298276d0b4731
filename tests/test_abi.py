"""The C-ABI library loads and exports every declared entry point; host-side
argument checks behave as documented.  No GPU needed."""
import ctypes

import pytest

from paper_1708_00720_b300 import xengine as xe


def test_every_declared_function_is_exported():
    names = xe.header_functions()
    assert len(names) >= 13
    lib = xe.library()
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings():
    for s in range(10):
        assert xe.xe_status_string(s) and xe.xe_status_string(s) != "unknown status"
    assert xe.xe_status_string(99) == "unknown status"
    assert "sm_103a" in xe.xe_version()


def _create(n, c, t, op=0, out=0):
    plan = ctypes.c_void_p()
    st = xe.status_of("xe_plan_create", ctypes.byref(plan), n, c, t, op, out)
    return st, plan


def test_create_argument_checks_before_touching_the_device():
    assert _create(20, 4, 16)[0] == xe.XE_ERR_ALIGNMENT
    assert _create(0, 4, 16)[0] == xe.XE_ERR_INVALID_ARG
    assert _create(16, 0, 16)[0] == xe.XE_ERR_INVALID_ARG
    assert _create(16, 4, 0)[0] == xe.XE_ERR_INVALID_ARG
    assert _create(16, 4, 16, op=7)[0] == xe.XE_ERR_INVALID_ARG
    assert _create(16, 4, 16, out=5)[0] == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_plan_create", None, 16, 4, 16, 0, 0) == xe.XE_ERR_INVALID_ARG


def test_create_without_gpu_fails_cleanly(gpu_available):
    if gpu_available:
        pytest.skip("a GPU is present")
    st, plan = _create(16, 4, 16)
    assert st in (xe.XE_ERR_CUDA, xe.XE_ERR_DEVICE_UNSUPPORTED)
    assert plan.value is None


def test_null_plan_calls_are_rejected():
    P = ctypes.c_void_p
    assert xe.status_of("xe_correlate", None, P(16), 1, 0, None) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_integrate", None, P(16), None) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_reset", None, None) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_unpack", None, P(16), P(16), 1, None) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_plan_check", None) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_plan_destroy", None) == xe.XE_OK
    out = ctypes.c_longlong()
    assert xe.status_of("xe_samples_integrated", None, ctypes.byref(out)) == xe.XE_ERR_INVALID_ARG


def test_product_package_does_not_import_the_oracle():
    import pathlib
    pkg = pathlib.Path(xe.__file__).parent
    for f in list(pkg.glob("*.py")) + list(pkg.glob("csrc/*")):
        text = f.read_text()
        assert "import oracle" not in text and "from oracle" not in text, f
        assert "xcorr_oracle" not in text, f


def test_calib_argument_checks_before_touching_the_device():
    h = ctypes.c_void_p()
    assert xe.status_of("xe_calib_create", ctypes.byref(h), 0, 4) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_calib_create", ctypes.byref(h), 8193, 4) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_calib_create", ctypes.byref(h), 16, 0) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_calib_create", None, 16, 4) == xe.XE_ERR_INVALID_ARG
    P = ctypes.c_void_p
    args = (P(16), P(16), P(16), None, 1)
    assert xe.status_of("xe_calib_chisq", None, *args, P(16), None) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_calib_grad", None, *args, None, P(16), None) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_calib_chisq_grad", None, *args, P(16), P(16), None) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_calib_scale", None, P(16), P(16), P(16), None) == xe.XE_ERR_INVALID_ARG
    assert xe.status_of("xe_calib_destroy", None) == xe.XE_OK
