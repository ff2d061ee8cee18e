"""The eq. 15 fit (Sec. 5) on data with a known answer.

- Synthetic ratios generated from the model itself are fitted exactly (log mu,
  gamma and c recovered to rounding), with and without log mu fixed.
- A mistake in the model (a dropped (gamma - 1) term, or 1/n in place of
  log(1 + 1/n)) would leave a residual and fail the first test.
- On the exact square-lattice counts c_1..c_16, the fit lands near the known
  growth constant (log mu_2 = 0.97008...): a loose but independent check, since
  the ratios of short square-lattice walks oscillate between even and odd n.
"""
import math

import numpy as np

from paper_2002_03000_gb300.analysis import fit_eq15, t_m
from tests.conftest import load_counts


def _synthetic(log_mu, gamma, c, n_max):
    lc = np.zeros(n_max + 1)
    for n in range(1, n_max):
        lc[n + 1] = lc[n] + log_mu + (gamma - 1.0) * math.log1p(1.0 / n) + c / (n * n)
    lc[1] = 0.0
    return lc


def test_fit_recovers_model_parameters():
    lc = _synthetic(1.5441609707, 1.15698, -0.37, 300)
    rv = np.full(lc.shape, 1e-8)
    f = fit_eq15(lc, rv, n_min=5)
    assert abs(f["log_mu"] - 1.5441609707) < 1e-9
    assert abs(f["gamma"] - 1.15698) < 1e-7
    assert abs(f["c"] + 0.37) < 1e-6
    g = fit_eq15(lc, rv, n_min=5, log_mu=1.5441609707)
    assert abs(g["gamma"] - 1.15698) < 1e-9 and abs(g["c"] + 0.37) < 1e-7


def test_fit_on_exact_square_counts():
    cn = load_counts(2)
    lc = np.log(np.array(cn, dtype=float))
    f = fit_eq15(lc, np.zeros(len(cn)), n_min=4)
    assert abs(f["log_mu"] - 0.970081) < 0.03, f


def test_t_m_is_mean_abs_log_error_over_lengths_1_to_M():
    best = np.log([1.0, 4.0, 12.0, 36.0])
    assert t_m(best, best) == 0.0
    est = best + np.array([5.0, 0.03, -0.06, 0.0])      # n = 0 does not count
    assert abs(t_m(est, best) - 0.03) < 1e-15
