"""Pins of the oracle's original PERM with cut-offs (Sec. 2: enrich into copies
above T_k, prune with probability 1 - 1/q below t_k).

Each branch is pinned by a special case whose outcome the mathematics fixes:
no cut-off active is the Rosenbluth method; always enriching grows a
deterministic tree at short lengths; always pruning makes survival a binomial
draw with an exactly known reweighting.  With both cut-offs active the
estimates obey the counting theorem against exact c_n."""
import math

import numpy as np
import pytest

from oracle import oracle as orc


def _scale(d, n):
    return 2.0 ** -orc.scale_exp(d, n)


def _cuts(d, n_max, hi, lo):
    return (np.array([hi(n) for n in range(n_max + 1)], dtype=float),
            np.array([lo(n) for n in range(n_max + 1)], dtype=float))


@pytest.mark.parametrize("d,n_max", [(2, 12), (3, 9)])
def test_no_cutoff_active_is_rosenbluth(d, n_max, exact_counts):
    """T = inf, t = 0: one walk per tour (no copies, no pruning), exact c_0..c_3,
    and the Rosenbluth estimator is unbiased (Sec. 1, eq. 3)."""
    h = orc.Oracle(d, n_max, 4, seed=21)
    hi, lo = _cuts(d, n_max, lambda n: math.inf, lambda n: 0.0)
    h.set_cutoffs(hi, lo, copies=2, q=2.0)
    h.run(2000)
    t = h.tables()
    M = 8000
    assert t["max_stack"] == 0
    assert np.all(t["S"] <= M)
    # a square-lattice walk cannot be trapped before 7 steps, a cubic one before 11
    assert np.all(t["S"][: min(n_max, 6) + 1] == M)
    lc, S, rv = h.estimates()
    for n in range(4):
        assert math.isclose(math.exp(lc[n]), exact_counts[d][n], rel_tol=1e-12)
    ex = np.array(exact_counts[d][: n_max + 1], dtype=float)
    z = (np.exp(lc - np.log(ex)) - 1.0)[4:] / np.sqrt(rv[4:])
    assert np.max(np.abs(z)) < 4.5, z


@pytest.mark.parametrize("copies", [2, 3])
def test_always_enrich_grows_a_fixed_tree(copies):
    """T = 0: every node past the empty walk makes min(copies, a_+) copies with
    distinct steps.  On the square lattice a_+ = 3 at lengths 1 and 2, so a tour
    has exactly 1, copies, copies^2 samples at lengths 1, 2, 3, and its weights
    there still sum to c_2 = 12 and c_3 = 36 exactly."""
    d, n_max, tours = 2, 3, 50
    h = orc.Oracle(d, n_max, 1, seed=5)
    hi, lo = _cuts(d, n_max, lambda n: 0.0, lambda n: 0.0)
    h.set_cutoffs(hi, lo, copies=copies, q=2.0)
    h.run(tours)
    t = h.tables()
    assert list(t["S"]) == [tours, tours, copies * tours, copies * copies * tours]
    lc, S, rv = h.estimates()
    assert math.isclose(math.exp(lc[2]), 12.0, rel_tol=1e-12)
    assert math.isclose(math.exp(lc[3]), 36.0, rel_tol=1e-12)


@pytest.mark.parametrize("q", [2.0, 3.0, 4.0])
def test_always_prune_is_binomial_with_exact_reweighting(q):
    """t = inf: every node past the empty walk survives with probability 1/q and
    then carries q W.  The samples at length 2 are Binomial(M, 1/q); each weighs
    4.3.q exactly, so W_2 = S_2 . 12 . q at the stored scale, and E[c_2] = 12."""
    d, n_max, M = 2, 4, 40000
    h = orc.Oracle(d, n_max, 8, seed=77)
    hi, lo = _cuts(d, n_max, lambda n: math.inf, lambda n: math.inf)
    h.set_cutoffs(hi, lo, copies=2, q=q)
    h.run(M // 8)
    t = h.tables()
    p = 1.0 / q
    S2 = t["S"][2]
    assert t["S"][0] == M and t["S"][1] == M
    assert abs(S2 - M * p) < 5.0 * math.sqrt(M * p * (1 - p))
    w_one = 12.0 * q * _scale(d, 2)
    assert math.isclose(t["W"][2], S2 * w_one, rel_tol=1e-12)
    # two survivals to reach length 3
    assert abs(t["S"][3] - M * p * p) < 5.0 * math.sqrt(M * p * p * (1 - p * p))


@pytest.mark.parametrize("d,n_max,copies,q,f", [(2, 14, 2, 2.0, 1.2), (3, 10, 3, 3.0, 1.1)])
def test_counting_theorem_with_both_cutoffs(d, n_max, copies, q, f, exact_counts):
    """Cut-offs around the exact c_n (T_n = f c_n, t_n = c_n / f at the stored
    scale): enrichment and pruning both happen, and the estimates stay within
    4.5 sigma of the exact counts at every length."""
    ex = exact_counts[d]
    hi, lo = _cuts(d, n_max, lambda n: f * ex[n] * _scale(d, n), lambda n: ex[n] / f * _scale(d, n))
    h = orc.Oracle(d, n_max, 4, seed=303)
    h.set_cutoffs(hi, lo, copies=copies, q=q)
    h.run(1500)
    t = h.tables()
    M = 6000
    assert t["max_stack"] > 0                      # copies were made
    # before the first possible trap (7 steps on the square lattice, 11 on the cubic) only pruning
    # removes samples
    assert np.any(t["S"][1:7] < M)
    lc, S, rv = h.estimates()
    e = np.array(ex[: n_max + 1], dtype=float)
    z = (np.exp(lc - np.log(e)) - 1.0)[4:] / np.sqrt(rv[4:])
    assert np.max(np.abs(z)) < 4.5, z


def test_cutoffs_reject_bad_arguments_and_switch_back():
    h = orc.Oracle(2, 6, 1, seed=1)
    hi, lo = _cuts(2, 6, lambda n: 0.0, lambda n: 0.0)
    for copies, q in ((0, 2.0), (5, 2.0), (2, 0.5)):
        with pytest.raises(RuntimeError):
            h.set_cutoffs(hi, lo, copies=copies, q=q)
    h.set_cutoffs(hi, lo, copies=2, q=2.0)
    h.set_cutoffs(None, None)
    h.run(3)
    ref = orc.Oracle(2, 6, 1, seed=1)
    ref.run(3)
    assert np.array_equal(h.tables()["S"], ref.tables()["S"])


def _rosenbluth_moments(d, n_max):
    """By brute force over all n-step self-avoiding walks: their number, and the
    sums of W and W^3, W(omega) being the Rosenbluth weight prod_{j<n} a_+(omega_j).
    A Rosenbluth walk has probability 1/W, so E[W] = c_n, E[W^2] = sum W and
    E[W^4] = sum W^3."""
    steps = [tuple(1 if i == j // 2 and j % 2 == 0 else (-1 if i == j // 2 else 0) for i in range(d))
             for j in range(2 * d)]
    s0 = np.zeros(n_max + 1)
    s1 = np.zeros(n_max + 1)
    s3 = np.zeros(n_max + 1)

    def rec(path, seen, w):
        n = len(path) - 1
        s0[n] += 1.0
        s1[n] += w
        s3[n] += w * w * w
        if n == n_max:
            return
        end = path[-1]
        free = [tuple(e + s for e, s in zip(end, st)) for st in steps]
        free = [p for p in free if p not in seen]
        for p in free:
            seen.add(p)
            path.append(p)
            rec(path, seen, w * len(free))
            path.pop()
            seen.discard(p)

    origin = tuple([0] * d)
    rec([origin], {origin}, 1.0)
    return s0, s1, s3


@pytest.mark.parametrize("d,n_max,tours", [(2, 8, 6000), (3, 5, 6000)])
def test_rosenbluth_second_moment_is_exact(d, n_max, tours):
    """With no cut-off active every tour is one Rosenbluth walk, so the per-tour
    sums X_t(n) are single weights and Q_n / M estimates E[W^2] = sum W exactly
    (the brute-force sum over all walks); the mean square's own standard error
    follows from E[W^4] = sum W^3."""
    count, e2, e4 = _rosenbluth_moments(d, n_max)
    h = orc.Oracle(d, n_max, 4, seed=61)
    hi, lo = _cuts(d, n_max, lambda n: math.inf, lambda n: 0.0)
    h.set_cutoffs(hi, lo, copies=2, q=2.0)
    h.run(tours // 4)
    t = h.tables()
    M = float(t["M"][0])
    for n in range(1, n_max + 1):
        s = 2.0 ** orc.scale_exp(d, n)
        mean_w2 = t["Q"][n] * s * s / M            # per-tour X^2 at the true scale
        var_w2 = e4[n] - e2[n] ** 2                  # Var(W^2) = E[W^4] - E[W^2]^2
        se = math.sqrt(max(var_w2, 0.0) / M)
        assert abs(mean_w2 - e2[n]) <= 5.0 * se + 1e-9 * e2[n], (n, mean_w2, e2[n], se)
        # the brute force counts the walks as the enumerator does
        assert count[n] == float(orc.enumerate_cn(d, n_max)[n])
