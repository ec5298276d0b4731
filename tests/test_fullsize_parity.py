"""Full-size workloads compared with the CPU oracle over EVERY baseline.

The benchmark's workload (512 inputs, 256 channels, 8192 samples: the LWA-SV
array of section "LWA Sevilleta implementation") is correlated by the int64
triple-loop oracle once per module, in full, and every operand path's output
of the benchmark's launch configuration (the fused one-gulp call) is compared
with it element by element.  The 2048-input workload is compared in full on
16 of its 64 channels (every baseline of those channels; the oracle's cost
grows with N^2).  These cases take minutes of host time on the oracle, which
starts in a background thread as soon as they are collected
(tests/fullsize_oracle.py); `-m "gpu and not fullsize"` skips them.
"""
import numpy as np
import pytest

from tests import fullsize_oracle

pytestmark = [pytest.mark.gpu, pytest.mark.fullsize]


@pytest.fixture(scope="module")
def xe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_00720_b300 import xengine
    return xengine


def emit(xe, x, operand):
    import torch
    T, C, N = x.shape
    eng = xe.XEngine(N, C, T, operand, "ci32")
    g = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    v = eng.correlate_emit(g)
    torch.cuda.synchronize()
    eng.check()
    out = v.cpu().numpy()
    eng.close()
    del g, v
    return out


@pytest.fixture(scope="module")
def lwa():
    return fullsize_oracle.result("lwa")


@pytest.fixture(scope="module")
def large_n():
    return fullsize_oracle.result("large_n")     # 16 of the 64 channels


@pytest.mark.parametrize("operand", ["fp8", "int32", "fp16"])
def test_lwa_every_baseline(xe, lwa, operand):
    x, want = lwa
    got = emit(xe, x, operand)
    assert got.shape == want.shape
    bad = np.argwhere(np.any(got != want, axis=-1))
    assert bad.size == 0, f"{len(bad)} of {want.shape[0] * want.shape[1]} visibilities differ, first {bad[:5]}"


@pytest.mark.parametrize("operand", ["fp8", "fp16"])
def test_large_n_every_baseline_of_16_channels(xe, large_n, operand):
    x, chans, want = large_n
    got = emit(xe, x, operand)[chans]
    bad = np.argwhere(np.any(got != want, axis=-1))
    assert bad.size == 0, f"{len(bad)} of {want.shape[0] * want.shape[1]} visibilities differ, first {bad[:5]}"
