"""The observable estimator of Sec. 1, eq. 5 in the oracle, for the squared
end-to-end distance |omega_n|^2.

Pins (none uses the oracle's own arithmetic as the reference):
- exact sums over all walks from an independent pure-Python brute force
  (n <= 7 square, n <= 5 cubic), and closed forms for n <= 2: one step gives 1;
  two steps give 4 (straight, 2d walks) or 2 (bent, 2d(2d-2) walks);
- the ratio estimator R_n / W_n from a flatPERM run agrees with the exact mean
  <|omega_n|^2> = (sum over walks) / c_n for n <= 16 within 2% (its spread at
  this size is a few tenths of a percent; using the previous site, or |omega|
  instead of |omega|^2, is off by 20% or more);
- <|omega_1|^2> = 1 exactly in every run (every one-step walk has it).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as orc
from tests import inputs


def _brute_r2(d, n):
    steps = inputs.STEPS[d]
    tot = [0] * (n + 1)
    for k in range(n + 1):
        for seq in itertools.product(range(2 * d), repeat=k):
            pos = (0,) * d
            seen = {pos}
            ok = True
            for j in seq:
                pos = tuple(p + s for p, s in zip(pos, steps[j]))
                if pos in seen:
                    ok = False
                    break
                seen.add(pos)
            if ok:
                tot[k] += sum(p * p for p in pos)
    return tot


@pytest.mark.parametrize("d,n", [(2, 7), (3, 5)])
def test_enumerated_r2_matches_brute_force(d, n):
    c, r2 = orc.enumerate_r2(d, n)
    assert list(r2) == _brute_r2(d, n)
    assert list(c) == list(orc.enumerate_cn(d, n))


@pytest.mark.parametrize("d", [2, 3])
def test_enumerated_r2_closed_forms(d):
    c, r2 = orc.enumerate_r2(d, 2)
    z = 2 * d
    assert r2[0] == 0 and r2[1] == z
    assert r2[2] == 4 * z + 2 * z * (z - 2)


@pytest.mark.parametrize("d,n_max,N,tours", [(2, 16, 12, 3000), (3, 11, 12, 1500)])
def test_ratio_estimator_matches_exact_mean(d, n_max, N, tours):
    c, r2 = orc.enumerate_r2(d, n_max)
    exact = r2 / c.astype(float)
    o = orc.Oracle(d, n_max, N, seed=4)
    o.run(tours)
    est = o.mean_r2()
    assert math.isclose(est[1], 1.0, rel_tol=1e-12)
    rel = np.abs(est[1:] / exact[1:] - 1.0)
    assert np.max(rel) < 0.02, rel
