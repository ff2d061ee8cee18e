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
import pytest

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


def test_alg1_combinations_on_oracle_tables(exact_counts):
    """Arithmetic: the oracle's own Algorithm-1 estimate.  Geometric: never above
    it, equal for one sequence, and exact where every sequence is exact (n <= 3:
    a sequential sequence's short lengths carry equal weights)."""
    import math
    from oracle import oracle as orc
    from paper_2002_03000_gb300 import analysis
    h = orc.Oracle(2, 14, 6, seed=4, alg=orc.ORC_ALG1)
    h.run(40)
    t = h.tables()
    lo, _, _ = h.estimates()
    ar = analysis.alg1_combine(t, 2, "arithmetic")
    ge = analysis.alg1_combine(t, 2, "geometric")
    assert np.allclose(ar, lo, rtol=1e-13, atol=1e-12)
    assert np.all(ge <= ar + 1e-12)
    for n in range(4):
        assert math.isclose(math.exp(ge[n]), exact_counts[2][n], rel_tol=1e-12)
    one = orc.Oracle(2, 10, 1, seed=4, alg=orc.ORC_ALG1)
    one.run(30)
    t1 = one.tables()
    assert np.allclose(analysis.alg1_combine(t1, 2, "geometric"), analysis.alg1_combine(t1, 2, "arithmetic"),
                       rtol=0, atol=1e-12)
    with pytest.raises(ValueError):
        analysis.alg1_combine(t, 2, "harmonic")
