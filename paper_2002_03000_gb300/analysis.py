"""Analysis of the estimates (host side): the growth constant from c_n ratios.

Sec. 5, eq. 15: log(c_{n+1}/c_n) ~ log mu_d + (gamma - 1) log(1 + 1/n) + c/n^2.
A three-parameter least-squares fit of that model to the estimated ratios over
n_min <= n < n_max, each ratio weighted by the inverse of its variance
(var(log c_{n+1}) + var(log c_n), the relative variances the library returns),
gives log mu_d, gamma and c.  With log mu_d fixed, the same fit has two
parameters (gamma, c).  This is post-processing of the tables the kernels
fill, not part of the growth path.
"""
from __future__ import annotations

import numpy as np


def fit_eq15(log_cn, relvar_n, n_min, n_max=None, log_mu=None):
    """Weighted fit of eq. 15.  log_cn, relvar_n: arrays indexed by n (as from
    perm_estimates).  Returns dict(log_mu, gamma, c, log_mu_err, gamma_err,
    n_min, n_max, points).  With log_mu given, only gamma and c are fitted."""
    lc = np.asarray(log_cn, dtype=float)
    rv = np.asarray(relvar_n, dtype=float)
    if n_max is None:
        n_max = len(lc) - 1
    n = np.arange(n_min, n_max, dtype=float)
    y = lc[n_min + 1:n_max + 1] - lc[n_min:n_max]
    var = rv[n_min + 1:n_max + 1] + rv[n_min:n_max]
    ok = np.isfinite(y) & np.isfinite(var)
    n, y, var = n[ok], y[ok], var[ok]
    pos = var[var > 0]
    floor = pos.min() if pos.size else 1.0
    w = 1.0 / np.maximum(var, floor)          # exact ratios (zero variance) get the largest weight
    x1 = np.log1p(1.0 / n)
    x2 = 1.0 / (n * n)
    if log_mu is None:
        A = np.stack([np.ones_like(n), x1, x2], axis=1)
        yy = y
    else:
        A = np.stack([x1, x2], axis=1)
        yy = y - log_mu
    sw = np.sqrt(w)
    coef, *_ = np.linalg.lstsq(A * sw[:, None], yy * sw, rcond=None)
    cov = np.linalg.pinv((A * w[:, None]).T @ A)
    err = np.sqrt(np.maximum(np.diag(cov), 0.0))
    if log_mu is None:
        return {"log_mu": float(coef[0]), "gamma": float(coef[1] + 1.0), "c": float(coef[2]),
                "log_mu_err": float(err[0]), "gamma_err": float(err[1]), "n_min": n_min,
                "n_max": n_max, "points": int(n.size)}
    return {"log_mu": float(log_mu), "gamma": float(coef[0] + 1.0), "c": float(coef[1]),
            "log_mu_err": 0.0, "gamma_err": float(err[0]), "n_min": n_min, "n_max": n_max,
            "points": int(n.size)}


def t_m(log_cn, log_best):
    """Sec. 4's convergence measure T_M: the mean over lengths n = 1..M of
    |log c_n(best) - log c_n(estimate)|, the total absolute error per unit
    length (M = the longest length with a best value)."""
    best = np.asarray(log_best, dtype=float)
    est = np.asarray(log_cn, dtype=float)[: len(best)]
    return float(np.mean(np.abs(best[1:] - est[1:])))


def alg1_combine(tables, d, mode="arithmetic"):
    """log c_n of an Algorithm-1 run from its per-sequence raw tables (the dict
    Run.tables() returns: W with one row of n_max+1 per sequence at the stored
    scale, M with each sequence's tours).

    arithmetic: the displayed estimator of Sec. 3, log of the mean over sequences
    of W_s/M_s (what perm_estimates returns);
    geometric: the mean over sequences of log(W_s/M_s), the combination Sec. 4
    uses for Algorithm 1's best estimate of log c_10000.  A length some sequence
    never reached gives -inf there.  By the inequality of arithmetic and geometric
    means the geometric form is never above the arithmetic one."""
    from . import _native
    M = np.asarray(tables["M"], dtype=np.int64).reshape(-1)
    N = M.size
    W = np.asarray(tables["W"], dtype=float).reshape(N, -1)
    if np.any(M < 1):
        raise ValueError("every sequence needs a tour")
    modes = {"arithmetic": _native.PERM_COMBINE_MEAN, "geometric": _native.PERM_COMBINE_GEOMETRIC}
    if mode not in modes:
        raise ValueError("mode is 'arithmetic' or 'geometric'")
    lc, _ = _native.perm_estimates_from_tables(d, W.shape[1] - 1, W, None, M, modes[mode])
    return lc
