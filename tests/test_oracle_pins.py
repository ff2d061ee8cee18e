"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these retypes the oracle's formulas: each checks a fact that an error
in the oracle (a dropped term, a wrong index or sign, a transposed operand)
would break -- published vectors, closed forms, an independent brute force,
exact invariants, probabilities and the Rosenbluth counting theorem.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from tests import inputs
from tests.conftest import GOLDEN


# --------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors (Salmon et al., SC'11)
# --------------------------------------------------------------------------
def test_philox_known_answers():
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            out = orc.philox4x32_10(v[0:4], v[4:6])
            assert list(out) == v[6:10]
            n += 1
    assert n == 3


# --------------------------------------------------------------------------
# Enumerator: closed forms, independent brute force, published leading terms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3])
def test_enumerate_closed_forms(d):
    c = orc.enumerate_cn(d, 4)
    z = 2 * d
    assert c[0] == 1
    assert c[1] == z
    assert c[2] == z * (z - 1)            # only the immediate reversal is forbidden
    assert c[3] == z * (z - 1) ** 2       # Z^d is bipartite: no 3-step return
    assert c[4] == z * (z - 1) ** 3 - z * (z - 2)   # minus the unit squares closed at step 4


def _brute_force(d, n):
    steps = inputs.STEPS[d]
    counts = [0] * (n + 1)
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
            counts[k] += ok
    return counts


@pytest.mark.parametrize("d,n", [(2, 7), (3, 5)])
def test_enumerate_matches_brute_force(d, n):
    assert list(orc.enumerate_cn(d, n)) == _brute_force(d, n)


def test_enumerate_leading_terms_published():
    with open(os.path.join(GOLDEN, "saw_leading_terms.txt")) as f:
        rows = [list(map(int, l.split())) for l in f if l.strip() and not l.startswith("#")]
    for d in (2, 3):
        nmax = max(n for dd, n, _ in rows if dd == d)
        c = orc.enumerate_cn(d, nmax)
        for dd, n, v in rows:
            if dd == d:
                assert c[n] == v


def test_golden_counts_are_enumerator_output(exact_counts):
    # the stored files are what the committed script writes
    assert list(orc.enumerate_cn(2, 16)) == exact_counts[2]
    assert list(orc.enumerate_cn(3, 11)) == exact_counts[3]


# --------------------------------------------------------------------------
# The ratio r of Sec. 2 (eq. 6): r = W / [W_n]^sample with the own weight in
# the running average.  Against the exact rational W M / (Wsum + W): three
# correctly rounded double operations stay within 2 ulp of it.  Special cases
# the paper fixes: a node whose own weight is the whole sum at its length has
# r = M (a first visit), and in particular r = 1 in the first tour (M = 1).
# --------------------------------------------------------------------------
def test_ratio_close_to_exact_definition():
    from fractions import Fraction
    rng = np.random.default_rng(5)
    for _ in range(4000):
        W = float(10.0 ** rng.uniform(-20, 20))
        M = int(rng.integers(1, 1 << 40))
        Wsum = 0.0 if rng.random() < 0.1 else float(W * M * 10.0 ** rng.uniform(-6, 6))
        r = orc.ratio(5, W, Wsum, M)
        exact = Fraction(W) * M / (Fraction(Wsum) + Fraction(W))
        assert abs(Fraction(r) - exact) <= Fraction(2 * 2.0 ** -52) * exact, (W, Wsum, M, r)
    assert orc.ratio(0, 3.0, 100.0, 7) == 1.0   # the empty walk always has r = 1


def test_ratio_first_visit_and_first_tour():
    rng = np.random.default_rng(6)
    for _ in range(2000):
        W = float(10.0 ** rng.uniform(-30, 30))
        assert orc.ratio(7, W, 0.0, 1) == 1.0            # first tour: own weight is all
        M = int(rng.integers(2, 1 << 30))
        r = orc.ratio(7, W, 0.0, M)                      # first visit: r = M
        assert abs(r - M) <= 2 * 2.0 ** -52 * M


# --------------------------------------------------------------------------
# One node on snapshot states
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3])
def test_step_a_plus_and_distinct_free_children(d):
    states = inputs.snapshot_batch(11 + d, d, 40, 300)
    for st in states:
        walk = st["walk"]
        n = walk.shape[0] - 1
        out = orc.step(d, 40, walk, st["W"], st["Wsum"], st["M"], st["ordinal"],
                       st["seq"], st["tour"], seed=77)
        free = inputs.free_neighbours(walk)
        if n == 40:
            assert out["outcome"] == 0
            continue
        assert out["a_plus"] == len(free)
        assert out["free_mask"] == sum(1 << j for j in free)
        if out["outcome"] == 3:
            assert 1 <= out["c"] <= out["a_plus"]
            assert len(set(out["dirs"])) == out["c"]            # distinct steps
            assert set(out["dirs"]) <= set(free)                # onto free sites only


def test_step_trapped_walk():
    trapped = inputs.shortest_trapped_walk_2d()     # independent geometric search
    assert trapped is not None and len(trapped) - 1 == 7   # shortest trap: 7 steps
    out = orc.step(2, 20, trapped, 1.0, 1.0, 10, 0, 0, 0, seed=1)
    assert out["outcome"] == 1 and out["a_plus"] == 0


@pytest.mark.parametrize("d", [2, 3])
def test_step_root(d):
    out = orc.step(d, 10, np.zeros((1, d), dtype=np.int32), 1.0, 123.0, 1000, 0, 3, 4, seed=9)
    assert out["outcome"] == 3 and out["a_plus"] == 2 * d and out["c"] == 1
    assert out["r"] == 1.0
    # the single child carries W a_+ = 2d at the stored scale of length 1
    assert out["child_w"] == 2 * d * 2.0 ** (-orc.scale_exp(d, 1))


def test_step_weight_conservation():
    """Enrichment conserves weight: c copies of W/c, each times a_+ (Sec. 2, eq. 2);
    a survivor of pruning carries W/r, r being its survival probability."""
    rng = np.random.default_rng(3)
    seen_enrich = seen_survive = 0
    for i in range(3000):
        d = 2 + (i % 2)
        n = int(rng.integers(1, 30))
        walk = inputs.random_saw(rng, d, n)
        st = inputs.random_state(rng, n)
        out = orc.step(d, 64, walk, st["W"], st["Wsum"], st["M"], st["ordinal"], st["seq"],
                       st["tour"], seed=1234)
        if out["outcome"] != 3:
            continue
        scale = 2.0 ** (orc.scale_exp(d, n + 1) - orc.scale_exp(d, n))
        a = out["a_plus"]
        if out["r"] >= 1.0:
            seen_enrich += 1
            total = out["c"] * out["child_w"] * scale
            assert abs(total - st["W"] * a) <= 4e-16 * st["W"] * a
        else:
            seen_survive += 1
            assert abs(out["child_w"] * scale * out["r"] - st["W"] * a) <= 8e-16 * st["W"] * a
    assert seen_enrich > 100 and seen_survive > 100


def test_step_enrichment_and_survival_probabilities():
    """P(c = floor r) = ceil(r) - r and P(survive) = r (Sec. 2), over many counters."""
    walk = np.array([[0, 0], [1, 0], [1, 1]], dtype=np.int32)   # a_+ = 3 at the end
    W = 1.0
    trials = 40000
    # Wsum chosen so that r = W M / (Wsum + W) is near the target
    for target in (2.3, 0.37):
        M = 1 << 30
        Wsum = M / target - 1.0
        counts = {}
        for k in range(trials):
            out = orc.step(2, 10, walk, W, Wsum, M, k, 1, 2, seed=99)
            key = out["c"] if out["outcome"] == 3 else 0
            counts[key] = counts.get(key, 0) + 1
        r = orc.ratio(2, W, Wsum, M)
        if target > 1:
            p = math.ceil(r) - r
            frac = counts.get(2, 0) / trials
            assert set(counts) <= {2, 3}
        else:
            p = r
            frac = counts.get(1, 0) / trials
            assert set(counts) <= {0, 1}
        sigma = math.sqrt(p * (1 - p) / trials)
        assert abs(frac - p) < 5 * sigma, (target, frac, p)


@pytest.mark.parametrize("c_target", [1, 2])
def test_step_direction_uniformity(c_target):
    """Children are a uniform choice of distinct free steps (Sec. 1: uniform choice)."""
    walk = np.array([[0, 0], [1, 0]], dtype=np.int32)   # free: +x, +y, -y (a_+ = 3)
    M = 1 << 30
    # c_target = 1: r = 1 exactly; c_target = 2: r = 2 exactly (p = 0)
    Wsum = M / c_target - 1.0
    counts = {}
    trials = 30000
    for k in range(trials):
        out = orc.step(2, 10, walk, 1.0, Wsum, M, k, 0, 0, seed=2024)
        assert out["c"] == c_target
        key = tuple(out["dirs"])
        counts[key] = counts.get(key, 0) + 1
    free = [0, 2, 3]
    cells = list(itertools.permutations(free, c_target))
    assert set(counts) == set(cells)
    expected = trials / len(cells)
    chi2 = sum((counts[c] - expected) ** 2 / expected for c in cells)
    dof = len(cells) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


# --------------------------------------------------------------------------
# Whole runs
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3])
def test_run_exact_short_lengths(d):
    """r = 1 at n = 0 and all weights at n <= 3 are equal, so in a sequential run
    c_0..c_3 come out exact and every tour visits each of these lengths once."""
    h = orc.Oracle(d, 12 if d == 2 else 9, 5, seed=31)
    h.run(300)
    lc, S, rv = h.estimates()
    M = h.tables()["M"][0]
    z = 2 * d
    for n, c in enumerate([1, z, z * (z - 1), z * (z - 1) ** 2]):
        assert math.isclose(math.exp(lc[n]), c, rel_tol=1e-12)
        assert S[n] == M


def test_run_first_tour_is_one_rosenbluth_chain():
    """With M = 1 and the own weight included, r = 1 at every node: the first tour
    grows a single walk with weight prod a_+ (Sec. 1, eq. 2)."""
    for seed in range(1, 30):
        h = orc.Oracle(2, 30, 1, seed=seed)
        h.run(1)
        t = h.tables()
        S = t["S"]
        n_end = int(np.max(np.nonzero(S)[0]))
        assert np.all(S[: n_end + 1] == 1) and np.all(S[n_end + 1:] == 0)
        assert t["steps"] == n_end + 1 and t["max_stack"] == 0
        # the weights are products of a_+ in 1..3 (2d at the root)
        for n in range(1, n_end + 1):
            w = t["W"][n] * 2.0 ** orc.scale_exp(2, n)
            assert w == round(w) and w >= 1


def _zscores(lc, rv, exact):
    ex = np.array(exact, dtype=float)
    rel = np.exp(lc[: len(ex)] - np.log(ex)) - 1.0
    with np.errstate(divide="ignore", invalid="ignore"):
        return rel / np.sqrt(rv[: len(ex)])


@pytest.mark.parametrize("d,n_max,alg", [(2, 16, 2), (3, 11, 2), (2, 16, 1)])
def test_run_counting_theorem(d, n_max, alg, exact_counts):
    """Sample averages of W_n estimate c_n (Sec. 1, eqs. 3-4): within 4 sigma."""
    h = orc.Oracle(d, n_max, 12, seed=1, alg=alg)
    h.run(4000)
    lc, S, rv = h.estimates()
    z = _zscores(lc, rv, exact_counts[d][: n_max + 1])
    zz = z[4:]
    assert np.all(np.isfinite(zz)) and np.max(np.abs(zz)) < 4.0, z


@pytest.mark.slow
def test_run_variance_calibration(exact_counts):
    """The per-tour variance estimate is calibrated: z-scores against exact c_n over
    independent seeds have unit spread."""
    zs = []
    for seed in range(40):
        h = orc.Oracle(2, 14, 4, seed=1000 + seed)
        h.run(1500)
        lc, S, rv = h.estimates()
        zs.append(_zscores(lc, rv, exact_counts[2][:15])[[6, 10, 14]])
    zs = np.array(zs)
    sd = zs.std(axis=0)
    mean = zs.mean(axis=0)
    assert np.all(sd > 0.6) and np.all(sd < 1.5), sd
    assert np.all(np.abs(mean) < 4 * sd / math.sqrt(len(zs))), mean


def test_run_cumulative_equals_single_call():
    a = orc.Oracle(2, 20, 3, seed=8)
    a.run(50)
    a.run(70)
    b = orc.Oracle(2, 20, 3, seed=8)
    b.run(120)
    ta, tb = a.tables(), b.tables()
    assert np.array_equal(ta["W"], tb["W"]) and np.array_equal(ta["S"], tb["S"])
    assert ta["M"][0] == tb["M"][0] == 360


def test_create_rejects_bad_arguments():
    for args in [(1, 10, 1), (4, 10, 1), (2, 0, 1), (2, 10, 0)]:
        with pytest.raises(ValueError):
            orc.Oracle(*args, seed=1)
