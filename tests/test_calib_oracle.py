"""Pins for the float64 gain-calibration oracle (no GPU): a hand-worked
single-input case, a zero-residual closed form, and central finite
differences of chi^2 -- which must reject deliberately broken gradients."""
import os

import numpy as np
import pytest

from oracle import calib
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "calib_hand_example.txt")


def read_hand():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, *v = line.split()
            vals[k] = [float(x) for x in v]
    g = np.array([[complex(*vals["g"])]])
    m = np.array([[complex(*vals["model"])]])
    v = np.array([[complex(*vals["vobs"])]])
    w = np.array([[vals["w"][0]]])
    return g, m, v, w, vals["chisq"][0], complex(*vals["grad"])


def random_problem(C=2, N=5, seed=0, weights=True):
    rng = np.random.default_rng(seed)
    nbl = N * (N + 1) // 2
    g = 1 + 0.3 * (rng.standard_normal((C, N)) + 1j * rng.standard_normal((C, N)))
    m = rng.standard_normal((C, nbl)) + 1j * rng.standard_normal((C, nbl))
    v = rng.standard_normal((C, nbl)) + 1j * rng.standard_normal((C, nbl))
    w = rng.uniform(0.5, 2.0, (C, nbl)) if weights else None
    return g, m, v, w


def fd_pin(grad_fn, g, m, v, w, include_autos=True, rtol=1e-6):
    fd = calib.finite_difference_grad(g, m, v, w, include_autos)
    an = grad_fn(g, m, v, w, include_autos)
    scale = max(abs(x) for x in fd.values())
    for (c, k), val in fd.items():
        assert abs(an[c, k] - val) <= rtol * scale, (c, k, an[c, k], val)


def test_hand_example():
    g, m, v, w, chi, gr = read_hand()
    assert calib.chisq(g, m, v, w) == pytest.approx(chi, rel=1e-15)
    assert calib.grad(g, m, v, w)[0, 0] == pytest.approx(gr, rel=1e-15)


def test_zero_residual():
    rng = np.random.default_rng(1)
    C, N = 3, 7
    g = 1 + 0.2 * (rng.standard_normal((C, N)) + 1j * rng.standard_normal((C, N)))
    m = synth.sky_model(N, C, seed=1)
    ii, jj = np.tril_indices(N)
    v = g[:, ii] * np.conj(g[:, jj]) * m
    assert calib.chisq(g, m, v) == pytest.approx(0.0, abs=1e-20)
    np.testing.assert_allclose(calib.grad(g, m, v), 0.0, atol=1e-12)


@pytest.mark.parametrize("include_autos", [True, False])
@pytest.mark.parametrize("weights", [True, False])
def test_gradient_matches_finite_differences(include_autos, weights):
    g, m, v, w = random_problem(weights=weights)
    fd_pin(calib.grad, g, m, v, w, include_autos)


def test_chisq_by_explicit_loop():
    g, m, v, w = random_problem(C=1, N=4, seed=3)
    total = 0.0
    p = 0
    for i in range(4):
        for j in range(i + 1):
            r = v[0, p] - g[0, i] * np.conj(g[0, j]) * m[0, p]
            total += w[0, p] * abs(r) ** 2
            p += 1
    assert calib.chisq(g, m, v, w) == pytest.approx(total, rel=1e-13)


def _broken_no_column_term(g, m, v, w=None, include_autos=True):
    gg = np.asarray(g, np.complex128)
    C, n = gg.shape
    ii, jj = np.tril_indices(n)
    r = calib.residuals(gg, m, v)
    ww = calib.weights(w, r.shape, include_autos, n)
    out = np.zeros((C, n), complex)
    for c in range(C):
        np.add.at(out[c], ii, (-ww * r * gg[:, jj] * np.conj(m))[c])
    return 2 * out


def _broken_missing_conj(g, m, v, w=None, include_autos=True):
    gg = np.asarray(g, np.complex128)
    C, n = gg.shape
    ii, jj = np.tril_indices(n)
    r = calib.residuals(gg, m, v)
    ww = calib.weights(w, r.shape, include_autos, n)
    out = np.zeros((C, n), complex)
    for c in range(C):
        np.add.at(out[c], ii, (-ww * r * gg[:, jj] * m)[c])
        np.add.at(out[c], jj, (-ww * np.conj(r) * gg[:, ii] * m)[c])
    return 2 * out


def _broken_factor(g, m, v, w=None, include_autos=True):
    return 0.5 * calib.grad(g, m, v, w, include_autos)


@pytest.mark.parametrize("broken", [_broken_no_column_term, _broken_missing_conj, _broken_factor])
def test_finite_differences_reject_broken_gradients(broken):
    g, m, v, w = random_problem(seed=4)
    with pytest.raises(AssertionError):
        fd_pin(broken, g, m, v, w)


@pytest.mark.parametrize("include_autos", [True, False])
def test_grad_entry_matches_finite_differences(include_autos):
    g, m, v, w = random_problem(C=2, N=6, seed=5)
    fd = calib.finite_difference_grad(g, m, v, w, include_autos)
    scale = max(abs(x) for x in fd.values())
    for (c, k), val in fd.items():
        assert abs(calib.grad_entry(g, m, v, w, include_autos, c, k) - val) <= 1e-6 * scale


def test_autos_only_single_input():
    # N = 1 leaves only the autocorrelation; without it chi^2 and grad vanish.
    g, m, v, w, chi, gr = read_hand()
    assert calib.chisq(g, m, v, w, include_autos=False) == 0.0
    assert calib.grad(g, m, v, w, include_autos=False)[0, 0] == 0.0


@pytest.mark.parametrize("include_autos", [True, False])
def test_input_part_of_chisq_carries_every_change(include_autos):
    # chi2 minus chisq_of_input(c, k) must not depend on g[c][k]: perturb it
    # and compare the two changes, and compare the derived central
    # differences with those of the whole chi2
    g, m, v, w = random_problem(C=2, N=9, seed=5)
    for (c, k) in [(0, 0), (1, 4), (0, 8), (1, 8)]:
        gp = g.copy()
        gp[c, k] += 0.37 - 0.21j
        full = calib.chisq(gp, m, v, w, include_autos) - calib.chisq(g, m, v, w, include_autos)
        part = (calib.chisq_of_input(gp, m, v, w, include_autos, c, k) -
                calib.chisq_of_input(g, m, v, w, include_autos, c, k))
        assert part == pytest.approx(full, rel=1e-12, abs=1e-12)
        fd_full = calib.finite_difference_grad(g, m, v, w, include_autos, index=[(c, k)])[(c, k)]
        fd_part = calib.finite_difference_entry(g, m, v, w, include_autos, c, k)
        assert abs(fd_part - fd_full) <= 1e-6 * abs(fd_full)
        assert abs(fd_part - calib.grad(g, m, v, w, include_autos)[c, k]) <= 1e-6 * abs(fd_full)


def test_input_part_rejects_a_dropped_column():
    # counting only row k (a plausible slip) misses terms that change with g_k
    g, m, v, w = random_problem(C=1, N=6, seed=6)
    c, k = 0, 2
    gp = g.copy()
    gp[c, k] += 0.5
    full = calib.chisq(gp, m, v, w) - calib.chisq(g, m, v, w)
    n = g.shape[1]
    ii, jj = np.tril_indices(n)
    row = ii == k
    r0 = calib.residuals(g, m, v)[0, row]
    r1 = calib.residuals(gp, m, v)[0, row]
    only_row = float(np.sum(w[0, row] * (np.abs(r1) ** 2 - np.abs(r0) ** 2)))
    assert abs(only_row - full) > 1e-6 * abs(full)
