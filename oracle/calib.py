"""Gain-calibration oracle in float64 -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, the smoke check and bench.py's CPU legs use this module;
the product library never imports it.

Model (applied to the X-engine's visibilities V_obs, per channel c and
baseline i >= j of the packed lower triangle, autocorrelations included):

    r_ij   = V_obs_ij - g_i conj(g_j) C_ij
    chi2   = sum_c sum_{i >= j} w_ij |r_ij|^2

and its gradient with respect to the complex gains, in the convention PyTorch
uses for a real loss of complex inputs (d/dRe g + i d/dIm g = 2 d/d conj(g)):

    d chi2 / d conj(g_k) = - sum_{j <= k} w_kj r_kj g_j conj(C_kj)
                           - sum_{i >= k} w_ik conj(r_ik) g_i C_ik

(both sums include the autocorrelation i = j = k).  The formula follows from
Wirtinger calculus treating g and conj(g) as independent: r_ij depends on
conj(g_j), conj(r_ij) on conj(g_i).  Pinned in tests/test_calib_oracle.py by
central finite differences of chi2, by a zero-residual closed form, and by a
single-baseline case worked by hand.

Arrays: g complex [C][N]; model, vobs complex [C][N(N+1)/2]; w real
[C][N(N+1)/2] or None (all ones).  `include_autos=False` drops i = j terms.
"""
from __future__ import annotations

import numpy as np


def tri_indices(n: int):
    """(i, j) of the packed lower triangle, in storage order."""
    return np.tril_indices(n)


def residuals(g: np.ndarray, model: np.ndarray, vobs: np.ndarray) -> np.ndarray:
    g = np.asarray(g, dtype=np.complex128)
    n = g.shape[-1]
    ii, jj = tri_indices(n)
    return np.asarray(vobs, np.complex128) - g[:, ii] * np.conj(g[:, jj]) * np.asarray(model, np.complex128)


def weights(w, shape, include_autos: bool, n: int) -> np.ndarray:
    ww = np.ones(shape, dtype=np.float64) if w is None else np.asarray(w, dtype=np.float64).copy()
    if not include_autos:
        ii, jj = tri_indices(n)
        ww[:, ii == jj] = 0.0
    return ww


def chisq(g, model, vobs, w=None, include_autos: bool = True) -> float:
    r = residuals(g, model, vobs)
    ww = weights(w, r.shape, include_autos, np.asarray(g).shape[-1])
    return float(np.sum(ww * (r.real ** 2 + r.imag ** 2)))


def grad(g, model, vobs, w=None, include_autos: bool = True) -> np.ndarray:
    """d chi2/d Re g + i d chi2/d Im g, complex [C][N]."""
    g = np.asarray(g, dtype=np.complex128)
    C, n = g.shape
    ii, jj = tri_indices(n)
    r = residuals(g, model, vobs)
    ww = weights(w, r.shape, include_autos, n)
    m = np.asarray(model, np.complex128)
    row_terms = -ww * r * g[:, jj] * np.conj(m)          # belongs to k = i
    col_terms = -ww * np.conj(r) * g[:, ii] * m          # belongs to k = j
    out = np.zeros((C, n), dtype=np.complex128)
    for c in range(C):
        np.add.at(out[c], ii, row_terms[c])
        np.add.at(out[c], jj, col_terms[c])
    return 2.0 * out


def grad_entry(g, model, vobs, w, include_autos: bool, c: int, k: int) -> complex:
    """One entry grad[c][k], summed straight from its two defining sums: row k
    of the triangle (baselines (k, j), j <= k) and column k (baselines (i, k),
    i >= k).  For sampled checks at sizes where grad() is too slow."""
    g = np.asarray(g[c], dtype=np.complex128)
    n = g.shape[0]
    total = 0j
    for j in range(k + 1):                      # row k: r_kj, term for g_k
        if j == k and not include_autos:
            continue
        p = k * (k + 1) // 2 + j
        m = complex(model[c][p])
        r = complex(vobs[c][p]) - g[k] * np.conj(g[j]) * m
        wt = 1.0 if w is None else float(w[c][p])
        total += -wt * r * g[j] * np.conj(m)
    for i in range(k, n):                       # column k: r_ik, term for g_k
        if i == k and not include_autos:
            continue
        p = i * (i + 1) // 2 + k
        m = complex(model[c][p])
        r = complex(vobs[c][p]) - g[i] * np.conj(g[k]) * m
        wt = 1.0 if w is None else float(w[c][p])
        total += -wt * np.conj(r) * g[i] * m
    return 2.0 * total


def finite_difference_grad(g, model, vobs, w=None, include_autos=True, step=1e-6, index=None):
    """Central differences of chi2 for selected (c, k) entries: returns
    {(c, k): dRe + i dIm}."""
    g = np.asarray(g, dtype=np.complex128)
    C, n = g.shape
    if index is None:
        index = [(c, k) for c in range(C) for k in range(n)]
    out = {}
    for (c, k) in index:
        parts = []
        for d in (step, 1j * step):
            gp = g.copy()
            gm = g.copy()
            gp[c, k] += d
            gm[c, k] -= d
            parts.append((chisq(gp, model, vobs, w, include_autos) -
                          chisq(gm, model, vobs, w, include_autos)) / (2 * step))
        out[(c, k)] = parts[0] + 1j * parts[1]
    return out


def chisq_of_input(g, model, vobs, w, include_autos: bool, c: int, k: int) -> float:
    """The part of chi2 that involves g[c][k]: the terms of baselines (k, j),
    j <= k (row k, autocorrelation included) and (i, k), i > k (column k below
    the diagonal), each counted once.  The rest of chi2 does not depend on
    g[c][k], so central differences of this part in g[c][k] equal those of
    chi2 itself, without the cancellation of a sum over every baseline."""
    gc = np.asarray(g[c], dtype=np.complex128)
    n = gc.shape[0]
    j = np.arange(k + 1)
    i = np.arange(k + 1, n)
    p = np.concatenate([k * (k + 1) // 2 + j, i * (i + 1) // 2 + k])
    gi = np.concatenate([np.full(k + 1, gc[k]), gc[i]])
    gj = np.concatenate([gc[j], np.full(n - k - 1, gc[k])])
    m = np.asarray(model[c], np.complex128)[p]
    r = np.asarray(vobs[c], np.complex128)[p] - gi * np.conj(gj) * m
    ww = np.ones(p.shape) if w is None else np.asarray(w[c], np.float64)[p]
    if not include_autos:
        ww = np.where(p == k * (k + 1) // 2 + k, 0.0, ww)
    return float(np.sum(ww * (r.real ** 2 + r.imag ** 2)))


def finite_difference_entry(g, model, vobs, w, include_autos: bool, c: int, k: int,
                            step: float = 1e-6) -> complex:
    """Central differences of chi2 in Re g[c][k] and Im g[c][k] (through
    chisq_of_input): dRe + i dIm."""
    g = np.array(g, dtype=np.complex128)
    parts = []
    for d in (step, 1j * step):
        g0 = g[c, k]
        g[c, k] = g0 + d
        fp = chisq_of_input(g, model, vobs, w, include_autos, c, k)
        g[c, k] = g0 - d
        fm = chisq_of_input(g, model, vobs, w, include_autos, c, k)
        g[c, k] = g0
        parts.append((fp - fm) / (2 * step))
    return parts[0] + 1j * parts[1]
