"""Fitting the paper's models to measured scan timings (host-side analysis).

Bandwidth-fraction law (§2, Eq. 2):  f = min(1, T_dec * b / (8 * beta)),
ridge b* = 8 * beta / T_dec.  T_dec is values/s, beta bytes/s, b bits.
§5 fits one T_dec per (machine, strategy); the paper does not say how, so
the fit here minimises the median absolute error |f - f_hat| over all
measured points by a 1-D search in log T (the paper reports exactly that
error), with a least-squares fit reported beside it.

Branch crossover (§6): branchy time A + B*sigma*(1 - sigma) against the
constant predicated cost C; branch-free wins where sigma*(1 - sigma) >
(C - A)/B = k, i.e. between sigma = (1 -+ sqrt(1 - 4k))/2.  On SIMT
hardware the divergence analogue replaces sigma*(1 - sigma) with
P_div(sigma) = 1 - sigma^32 - (1 - sigma)^32, the probability that a
32-value warp group mixes matches and misses (i.i.d. data).
"""
from __future__ import annotations

import math

import numpy as np


def law_f(t_dec, b, beta):
    """Predicted bandwidth fraction for width(s) b."""
    return np.minimum(1.0, np.asarray(t_dec, dtype=float) * np.asarray(b, dtype=float) / (8.0 * beta))


def ridge(t_dec, beta):
    """Width b* at which decode stops limiting the scan."""
    return 8.0 * beta / t_dec


def implied_beta(t_dec, b_star):
    """Bandwidth implied by a (T_dec, b*) pair: beta = b* * T_dec / 8."""
    return b_star * t_dec / 8.0


def _median_err(t, b, f, beta):
    return float(np.median(np.abs(f - law_f(t, b, beta))))


def _objective(t, b, f, beta):
    # the median is flat once most widths sit on the plateau f = 1; a small
    # RMS term picks one T_dec among the equally good ones
    r = f - law_f(t, b, beta)
    return float(np.median(np.abs(r))) + 1e-3 * float(np.sqrt(np.mean(r * r)))


def fit_tdec(b, f, beta, lo=1e6, hi=1e15):
    """T_dec minimising median |f - f_hat|; returns (T_dec, median error).

    Coarse log-grid search, then golden-section refinement around the best
    grid point (the objective is piecewise smooth in log T)."""
    b = np.asarray(b, dtype=float)
    f = np.asarray(f, dtype=float)
    grid = np.exp(np.linspace(math.log(lo), math.log(hi), 4001))
    errs = np.array([_objective(t, b, f, beta) for t in grid])
    i = int(np.argmin(errs))
    a = math.log(grid[max(i - 1, 0)])
    c = math.log(grid[min(i + 1, grid.size - 1)])
    g = (math.sqrt(5) - 1) / 2
    x1, x2 = c - g * (c - a), a + g * (c - a)
    e1, e2 = _objective(math.exp(x1), b, f, beta), _objective(math.exp(x2), b, f, beta)
    for _ in range(80):
        if e1 <= e2:
            c, x2, e2 = x2, x1, e1
            x1 = c - g * (c - a)
            e1 = _objective(math.exp(x1), b, f, beta)
        else:
            a, x1, e1 = x1, x2, e2
            x2 = a + g * (c - a)
            e2 = _objective(math.exp(x2), b, f, beta)
    best_t = min((errs[i], grid[i]), (e1, math.exp(x1)), (e2, math.exp(x2)))[1]
    return float(best_t), _median_err(best_t, b, f, beta)


def fit_tdec_lsq(b, f, beta, lo=1e6, hi=1e15):
    """Least-squares T_dec (same search, squared error)."""
    b = np.asarray(b, dtype=float)
    f = np.asarray(f, dtype=float)
    grid = np.exp(np.linspace(math.log(lo), math.log(hi), 20001))
    sse = np.array([float(np.sum((f - law_f(t, b, beta)) ** 2)) for t in grid])
    i = int(np.argmin(sse))
    return float(grid[i]), float(math.sqrt(sse[i] / max(b.size, 1)))


def band_edges(k):
    """Selectivities where sigma*(1-sigma) = k; None if the parabola never reaches k."""
    if k > 0.25:
        return None
    if k <= 0:
        return (0.0, 1.0)
    r = math.sqrt(1.0 - 4.0 * k)
    return ((1.0 - r) / 2.0, (1.0 + r) / 2.0)


def p_div(sigma, group=32):
    """Probability that a group of `group` i.i.d. values mixes matches and misses."""
    s = np.asarray(sigma, dtype=float)
    return 1.0 - s ** group - (1.0 - s) ** group


def fit_affine(x, y):
    """Least squares y = A + B x; returns (A, B)."""
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    m = np.vstack([np.ones_like(x), x]).T
    (a, bcoef), *_ = np.linalg.lstsq(m, y, rcond=None)
    return float(a), float(bcoef)


def fit_branch_models(sigma, t_branchy, t_branchfree):
    """Fit the parabola and the divergence model to branchy times.

    Returns a dict with both fits, the constant predicated cost C and the
    band in which branch-free wins under the parabola model."""
    s = np.asarray(sigma, dtype=float)
    tb = np.asarray(t_branchy, dtype=float)
    c = float(np.mean(np.asarray(t_branchfree, dtype=float)))
    a1, b1 = fit_affine(s * (1 - s), tb)
    a2, b2 = fit_affine(p_div(s), tb)
    edges = band_edges((c - a1) / b1) if b1 > 0 else None
    return {
        "C_branchfree": c,
        "parabola": {"A": a1, "B": b1, "band_branchfree_wins": edges},
        "divergence": {"A": a2, "B": b2},
    }
