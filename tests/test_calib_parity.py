"""GPU gain calibration (chi^2 and its adjoint) vs the float64 oracle.

The kernels compute every per-baseline term in float32 from float32 inputs,
so the comparison is against the oracle evaluated on the same float32 values
(widened to float64), with tolerances derived from that arithmetic
(u = 2^-24, the float32 unit roundoff):

* chi^2: each term w |r|^2 has error at most about 2|r||dr| + 4u|r|^2 with
  |dr| <= u|r| + 6u M, M = |g_i||g_j||C_ij| (two complex products and a
  subtraction); the Kahan/float64 sums add at most 2u chi^2.  Bound used:
  16 u sum w (|r| M + |r|^2).  The relative error must also be <= 1e-6.
* gradient entry k: n_k terms w r g conj(C) (or its column twin), each with
  error <= 6u w |g||C| (|r| + M), summed in float32 in chains of at most n_k
  additions.  Bound used: 2 u (n_k + 8) A_k, A_k = sum over the entry's
  terms of w |g||C| (|r| + M).  The normwise relative error must also be
  <= 1e-5.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import calib as ocal

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def cal():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_00720_b300 import calib
    return calib


def problem(C, N, seed, weights=True, vobs=None):
    rng = np.random.default_rng(seed)
    nbl = N * (N + 1) // 2
    g = synth.gains(N, C, seed).astype(np.complex64)
    m = synth.sky_model(N, C, seed).astype(np.complex64)
    if vobs is None:
        vobs = (m * (1 + 0.3 * rng.standard_normal((C, nbl))) +
                2 * (rng.standard_normal((C, nbl)) + 1j * rng.standard_normal((C, nbl))))
    v = np.asarray(vobs).astype(np.complex64)
    w = rng.uniform(0.5, 2.0, (C, nbl)).astype(np.float32) if weights else None
    return g, m, v, w


def magnitudes(g, m, v, w, include_autos):
    """|r|, M and the effective weights, in float64."""
    gg = g.astype(np.complex128)
    N = g.shape[1]
    ii, jj = np.tril_indices(N)
    r = ocal.residuals(gg, m, v)
    M = np.abs(gg[:, ii]) * np.abs(gg[:, jj]) * np.abs(m.astype(np.complex128))
    ww = ocal.weights(w, r.shape, include_autos, N)
    return np.abs(r), M, ww, ii, jj


def chisq_tol(g, m, v, w, include_autos):
    ar, M, ww, _, _ = magnitudes(g, m, v, w, include_autos)
    return 16 * U * float(np.sum(ww * (ar * M + ar * ar)))


def grad_tol(g, m, v, w, include_autos):
    ar, M, ww, ii, jj = magnitudes(g, m, v, w, include_autos)
    C, N = g.shape
    ag = np.abs(g.astype(np.complex128))
    am = np.abs(m.astype(np.complex128))
    row = ww * ag[:, jj] * am * (ar + M)     # terms of g_i
    col = ww * ag[:, ii] * am * (ar + M)     # terms of g_j
    A = np.zeros((C, N))
    for c in range(C):
        np.add.at(A[c], ii, row[c])
        np.add.at(A[c], jj, col[c])
    n = N + 1
    return 2 * U * (n + 8) * A


def to_dev(*arrs):
    import torch
    return [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def check_chisq(got, g, m, v, w, include_autos, relative=True):
    """Derived bound always; the relative 1e-6 only where chi^2 is not itself
    a cancellation residue (relative=False for a fit that is exact up to the
    float32 rounding of V)."""
    ref = ocal.chisq(g, m, v, w, include_autos)
    assert abs(got - ref) <= chisq_tol(g, m, v, w, include_autos) + 1e-300, (got, ref)
    if relative:
        assert abs(got - ref) <= 1e-6 * abs(ref) + 1e-30
    return ref


def check_grad(got, g, m, v, w, include_autos, scale=1.0, relative=True):
    ref = scale * ocal.grad(g, m, v, w, include_autos)
    tol = abs(scale) * grad_tol(g, m, v, w, include_autos)
    err = np.abs(got.astype(np.complex128) - ref)
    bad = np.argwhere(err > tol + 1e-30)
    assert bad.size == 0, (bad[:5], err[tuple(bad[0])], tol[tuple(bad[0])])
    nref = np.linalg.norm(ref)
    if relative and nref > 0:
        assert np.linalg.norm(got - ref) <= 1e-5 * nref


SHAPES = [(3, 1), (2, 5), (3, 32), (2, 33), (1, 64), (2, 100), (1, 257)]


@pytest.mark.parametrize("include_autos", [True, False])
@pytest.mark.parametrize("weights", [True, False])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"C{s[0]}N{s[1]}")
def test_chisq_and_grad(cal, shape, weights, include_autos):
    import torch
    C, N = shape
    g, m, v, w = problem(C, N, seed=N + 7 * C, weights=weights)
    dg, dm, dv, dw = to_dev(g, m, v, w)
    k = cal.Calibrator(N, C)
    chi = k.chisq(dg, dm, dv, dw, include_autos)
    grad = k.grad(dg, dm, dv, dw, include_autos)
    chi2, grad2 = k.chisq_grad(dg, dm, dv, dw, include_autos)
    torch.cuda.synchronize()
    check_chisq(chi.item(), g, m, v, w, include_autos)
    check_chisq(chi2.item(), g, m, v, w, include_autos)
    check_grad(grad.cpu().numpy(), g, m, v, w, include_autos)
    check_grad(grad2.cpu().numpy(), g, m, v, w, include_autos)
    k.close()


def test_hand_example_on_gpu(cal):
    import torch
    g = torch.tensor([[1 + 1j]], dtype=torch.complex64, device="cuda")
    m = torch.tensor([[2 + 0j]], dtype=torch.complex64, device="cuda")
    v = torch.tensor([[5 + 0j]], dtype=torch.complex64, device="cuda")
    k = cal.Calibrator(1, 1)
    chi, grad = k.chisq_grad(g, m, v, None, True)
    assert chi.item() == 1.0
    assert complex(grad.cpu()[0, 0]) == -8 - 8j


def test_zero_residual_gives_zero(cal):
    import torch
    C, N = 2, 40
    g = synth.gains(N, C, 3).astype(np.complex64)
    m = synth.sky_model(N, C, 3).astype(np.complex64)
    ii, jj = np.tril_indices(N)
    v = (g[:, ii].astype(np.complex128) * np.conj(g[:, jj]) * m).astype(np.complex64)
    dg, dm, dv = to_dev(g, m, v)
    k = cal.Calibrator(N, C)
    chi, grad = k.chisq_grad(dg, dm, dv, None, True)
    check_chisq(chi.item(), g, m, v, None, True, relative=False)
    check_grad(grad.cpu().numpy(), g, m, v, None, True, relative=False)
    assert chi.item() < 1e-6 * float(np.sum(np.abs(v.astype(np.complex128)) ** 2))


def test_scaled_gradient_and_autograd(cal):
    import torch
    C, N = 2, 70
    g, m, v, w = problem(C, N, seed=11)
    dg, dm, dv, dw = to_dev(g, m, v, w)
    k = cal.Calibrator(N, C)
    s = torch.tensor(-2.5, dtype=torch.float64, device="cuda")
    check_grad(k.grad(dg, dm, dv, dw, True, scale=s).cpu().numpy(), g, m, v, w, True, scale=-2.5)

    gp = dg.clone().requires_grad_(True)
    loss = 3.0 * cal.chisq(gp, dm, dv, dw, True, calibrator=k)
    loss.backward()
    check_chisq(loss.item() / 3.0, g, m, v, w, True)
    check_grad(gp.grad.cpu().numpy(), g, m, v, w, True, scale=3.0)

    with torch.no_grad():
        out = cal.chisq(dg, dm, dv, dw, False, calibrator=k)
    check_chisq(out.item(), g, m, v, w, False)


def test_gradient_descent_lowers_chisq(cal):
    import torch
    C, N = 4, 48
    rng = np.random.default_rng(5)
    g_true = synth.gains(N, C, 5, scatter=0.3)
    m = synth.sky_model(N, C, 5)
    ii, jj = np.tril_indices(N)
    v = g_true[:, ii] * np.conj(g_true[:, jj]) * m
    dm, dv = to_dev(m.astype(np.complex64), v.astype(np.complex64))
    g = torch.ones((C, N), dtype=torch.complex64, device="cuda", requires_grad=True)
    k = cal.Calibrator(N, C)
    opt = torch.optim.Adam([g], lr=0.02)
    first = None
    for _ in range(60):
        opt.zero_grad()
        loss = cal.chisq(g, dm, dv, None, True, calibrator=k)
        loss.backward()
        opt.step()
        first = first if first is not None else loss.item()
    assert loss.item() < 0.1 * first


def test_deterministic(cal):
    import torch
    C, N = 3, 300
    g, m, v, w = problem(C, N, seed=2)
    dg, dm, dv, dw = to_dev(g, m, v, w)
    k = cal.Calibrator(N, C)
    a = k.chisq_grad(dg, dm, dv, dw, True)
    b = k.chisq_grad(dg, dm, dv, dw, True)
    torch.cuda.synchronize()
    assert a[0].item() == b[0].item()
    assert torch.equal(torch.view_as_real(a[1]), torch.view_as_real(b[1]))


def test_argument_errors(cal):
    import ctypes
    import torch
    from paper_1708_00720_b300 import xengine as xe
    C, N = 2, 8
    g, m, v, w = problem(C, N, seed=1)
    dg, dm, dv, dw = to_dev(g, m, v, w)
    k = cal.Calibrator(N, C)
    with pytest.raises(ValueError):
        k.chisq(dg[:, :4].contiguous(), dm, dv, dw)
    with pytest.raises(ValueError):
        k.chisq(dg, dm.to(torch.complex128), dv, dw)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    raw = torch.view_as_real(dg)
    P = ctypes.c_void_p
    st = xe.status_of("xe_calib_chisq", k.handle, P(raw.data_ptr() + 4), P(torch.view_as_real(dm).data_ptr()),
                      P(torch.view_as_real(dv).data_ptr()), None, 1, P(out.data_ptr()), None)
    assert st == xe.XE_ERR_ALIGNMENT
    st = xe.status_of("xe_calib_chisq", k.handle, P(raw.data_ptr()), P(torch.view_as_real(dm).data_ptr()),
                      P(torch.view_as_real(dv).data_ptr()), None, 2, P(out.data_ptr()), None)
    assert st == xe.XE_ERR_INVALID_ARG
    st = xe.status_of("xe_calib_grad", k.handle, P(raw.data_ptr()), P(torch.view_as_real(dm).data_ptr()),
                      P(torch.view_as_real(dv).data_ptr()), None, 1, None, None, None)
    assert st == xe.XE_ERR_INVALID_ARG


@pytest.fixture(scope="module")
def calib_workload(cal):
    """512 inputs, 128 channels: V_obs from the oracle X-engine on the seeded
    voltages (64 samples, to keep the oracle fast), a sky model and random
    gains; the GPU's chi^2 and gradient of it."""
    import torch
    p = synth.CALIB_CONFIG
    N, C = p["n_input"], p["n_chan"]
    x = synth.voltages(N, C, 64, seed=p["seed"], random_phase=True)
    vi = oracle.correlate(x)
    vobs = (vi[..., 0] + 1j * vi[..., 1]).astype(np.complex64)
    g = synth.gains(N, C, p["seed"]).astype(np.complex64)
    m = synth.sky_model(N, C, p["seed"]).astype(np.complex64)
    w = np.ones(vobs.shape, np.float32)
    dg, dm, dv, dw = to_dev(g, m, vobs, w)
    k = cal.Calibrator(N, C)
    chi, grad = k.chisq_grad(dg, dm, dv, dw, True)
    torch.cuda.synchronize()
    out = (g, m, vobs, w, chi.item(), grad.cpu().numpy())
    k.close()
    return out


def test_calibration_workload_full_size(calib_workload):
    g, m, vobs, w, chi, grad = calib_workload
    ref = check_chisq(chi, g, m, vobs, w, True)
    check_grad(grad, g, m, vobs, w, True)
    want = ocal.grad(g, m, vobs, w, True)
    err = np.abs(grad.astype(np.complex128) - want)
    print(f"\ncalibration 512x128 vs the float64 oracle: chi^2 rel {abs(chi - ref) / ref:.3e}; "
          f"gradient max |err| / max |grad| {err.max() / np.abs(want).max():.3e}, "
          f"normwise {np.linalg.norm(err) / np.linalg.norm(want):.3e}")


def test_calibration_workload_gradient_vs_finite_differences(calib_workload):
    """The GPU gradient at 96 sampled (channel, input) entries against central
    float64 finite differences (step 1e-6) of the float64 chi^2 in Re g and
    Im g.  Only the baselines of input k change with g_k, so the differences
    are taken of that part of chi^2 (oracle.calib.chisq_of_input), free of the
    cancellation of the whole sum; chi^2 is quadratic in g_k except for the
    autocorrelation term, so the truncation error is negligible."""
    g, m, vobs, w, chi, grad = calib_workload
    C, N = g.shape
    rng = np.random.default_rng(11)
    idx = [(int(c), int(k)) for c, k in zip(rng.integers(0, C, 90), rng.integers(0, N, 90))]
    idx += [(0, 0), (0, N - 1), (C - 1, 0), (C - 1, N - 1), (5, 63), (5, 64)]
    tol = grad_tol(g, m, vobs, w, True)
    step = 1e-6
    fd = np.array([ocal.finite_difference_entry(g, m, vobs, w, True, c, k, step) for c, k in idx])
    got = np.array([grad[c, k] for c, k in idx]).astype(np.complex128)
    an = np.array([ocal.grad_entry(g, m, vobs, w, True, c, k) for c, k in idx])
    # rounding of a central difference: each of its float64 chi^2 parts errs
    # by at most ~16 * 2^-53 of itself (pairwise sums), divided by 2 step,
    # for the real and the imaginary direction
    part = np.array([ocal.chisq_of_input(g, m, vobs, w, True, c, k) for c, k in idx])
    fd_err = 2 * 16 * 2.0 ** -53 * part / (2 * step) * np.sqrt(2)
    assert np.all(np.abs(fd - an) <= fd_err + 1e-9 * np.abs(an))
    err = np.abs(got - fd)
    bound = np.array([tol[c, k] for c, k in idx]) + fd_err
    assert np.all(err <= bound), np.argwhere(err > bound)[:5]
    rel = err / np.abs(fd)
    normwise = np.linalg.norm(err) / np.linalg.norm(fd)
    assert rel.max() <= 1e-5 and normwise <= 1e-5, (rel.max(), normwise)
    print(f"\ncalibration 512x128, {len(idx)} entries vs float64 central differences: "
          f"max rel {rel.max():.3e}, normwise {normwise:.3e}")


def test_maximum_inputs_sampled(cal):
    """N = 8192 (the largest accepted), one channel: chi^2 in full, gradient
    entries sampled and computed one by one by the oracle."""
    import torch
    N, C = 8192, 1
    nbl = N * (N + 1) // 2
    rng = np.random.default_rng(9)
    g = synth.gains(N, C, 9).astype(np.complex64)
    m = (rng.standard_normal((C, nbl)) + 1j * rng.standard_normal((C, nbl))).astype(np.complex64)
    v = (rng.standard_normal((C, nbl)) + 1j * rng.standard_normal((C, nbl))).astype(np.complex64) * 4
    dg, dm, dv = to_dev(g, m, v)
    k = cal.Calibrator(N, C)
    chi, grad = k.chisq_grad(dg, dm, dv, None, True)
    torch.cuda.synchronize()
    ref = ocal.chisq(g, m, v, None, True)
    assert abs(chi.item() - ref) <= 1e-6 * ref
    got = grad.cpu().numpy()
    gg = g[0].astype(np.complex128)
    ks = [0, 1, 31, 32, 4095, 8160, 8191]
    ents = {kk: ocal.grad_entry(g, m, v, None, True, 0, kk) for kk in ks}
    rms = float(np.sqrt(np.mean([abs(e) ** 2 for e in ents.values()])))
    for kk, e in ents.items():
        # the same bound as grad_tol, for this entry's row and column only
        jr = np.arange(kk + 1)
        ic = np.arange(kk, N)
        pr = kk * (kk + 1) // 2 + jr
        pc = ic * (ic + 1) // 2 + kk
        A = 0.0
        for p_, gi, gj, go in ((pr, gg[kk], gg[jr], gg[jr]), (pc, gg[ic], gg[kk], gg[ic])):
            mm = m[0, p_].astype(np.complex128)
            r = v[0, p_] - gi * np.conj(gj) * mm
            M = np.abs(gi) * np.abs(gj) * np.abs(mm)
            A += float(np.sum(np.abs(go) * np.abs(mm) * (np.abs(r) + M)))
        assert abs(got[0, kk] - e) <= 2 * U * (N + 9) * A, (kk, got[0, kk], e)
        assert abs(got[0, kk] - e) <= 1e-5 * rms, (kk, got[0, kk], e)
