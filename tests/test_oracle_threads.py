"""The oracle's Algorithm 2 on several host threads (the paper's own form, Sec. 3),
timed as the CPU baseline: on one thread it is the sequential oracle exactly; on
several it keeps the exact short lengths and the counting theorem."""
import math

import numpy as np

from oracle import oracle as orc


def test_one_thread_is_the_sequential_run():
    a = orc.Oracle(2, 24, 5, seed=19)
    a.run(60)
    b = orc.Oracle(2, 24, 5, seed=19)
    b.run_threads(60, 1)
    ta, tb = a.tables(), b.tables()
    for k in ("W", "S", "Q"):
        assert np.array_equal(ta[k], tb[k]), k
    assert ta["M"][0] == tb["M"][0] == 300 and ta["steps"] == tb["steps"]


def test_threads_keep_exact_lengths_and_the_counting_theorem(exact_counts):
    for d, n_max in ((2, 16), (3, 11)):
        h = orc.Oracle(d, n_max, 12, seed=3)
        h.run_threads(3000, 4)
        t = h.tables()
        M = 12 * 3000
        assert t["M"][0] == M and t["S"][0] == M and t["S"][1] == M
        lc, S, rv = h.estimates()
        assert math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
        ex = np.array(exact_counts[d][: n_max + 1], dtype=float)
        z = (np.exp(lc - np.log(ex)) - 1.0)[2:] / np.sqrt(rv[2:] + 1e-10)
        assert np.max(np.abs(z)) < 4.5, z


def test_threads_reject_what_they_do_not_run():
    h = orc.Oracle(2, 8, 2, seed=1, alg=orc.ORC_ALG1)
    try:
        h.run_threads(1, 2)
        raise AssertionError("Algorithm 1 accepted")
    except RuntimeError:
        pass
