"""The oracle's pins are sensitive: plant plausible mistakes in a temporary copy
of the oracle source (on the CPU only), rebuild it, and check that at least one
pin fails for every mistake while all of them hold for the real source."""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import oracle as orc
from tests import inputs
from tests.conftest import load_counts

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "perm_oracle.c")

MUTATIONS = {
    "child weight misses a_+": ("o->child_w = ldexp(Wp * (double)a, -dE);",
                                "o->child_w = ldexp(Wp, -dE);"),
    "copies keep full weight": ("Wp = W / (double)c;                               /* each copy",
                                "Wp = W;                               /* each copy"),
    "survivor not reweighted": ("Wp = W * (1.0 / r);", "Wp = W;"),
    "survivor weight times r, not 1/r": ("Wp = W * (1.0 / r);", "Wp = W * r;"),
    "own weight left out of r": ("double avg = (Wsum + W) / (double)M;", "double avg = Wsum / (double)M;"),
    "M off by one": ("double avg = (Wsum + W) / (double)M;", "double avg = (Wsum + W) / (double)(M + 1);"),
    "running average not divided by M": ("double avg = (Wsum + W) / (double)M;", "double avg = Wsum + W;"),
    "ratio inverted": ("return W / avg;", "return avg / W;"),
    "rounding probability inverted": ("double c_raw = (u0 < p) ? fl : ce;",
                                      "double c_raw = (u0 < p) ? ce : fl;"),
    "rounding probability from the fraction": ("double p = ce - r;", "double p = r - fl;"),
    "survival with probability 1 - r": ("if (!(u0 < r)) return ORC_LEAF_PRUNED;",
                                        "if (!(u0 < 1.0 - r)) return ORC_LEAF_PRUNED;"),
    "Fisher-Yates offset dropped": ("int j = i + (int)(prod >> 32);", "int j = (int)(prod >> 32);"),
    "backtrack leaves a site": ("for (int k = n; k > dp; --k) occ_set(&h->occ",
                                "for (int k = n; k > dp + 1; --k) occ_set(&h->occ"),
    "variance from X not X^2": ("Qn[k] += h->X[k] * h->X[k];", "Qn[k] += h->X[k];"),
    "direction signs swapped": ("to[j >> 1] += (j & 1) ? -1 : 1;", "to[j >> 1] += (j & 1) ? 1 : -1;"),
    "scale step wrong": ("int dE = orc_scale_exp(d, n + 1) - orc_scale_exp(d, n);",
                         "int dE = orc_scale_exp(d, n + 1);"),
    "tour sum counts visits": ("h->X[n] += W;", "h->X[n] += 1.0;"),
    "root ratio not forced": ("if (n == 0) return 1.0;", "if (n < 0) return 1.0;"),
    "Philox round permutation": ("uint32_t y0 = hi1 ^ x1 ^ k0;", "uint32_t y0 = hi0 ^ x1 ^ k0;"),
    "observable at the previous site": ("const int64_t x = co[(long)n * d + i];",
                                        "const int64_t x = co[(long)(n > 0 ? n - 1 : 0) * d + i];"),
    "observable not squared": ("r2 += x * x;", "r2 += x < 0 ? -x : x;"),
    "observable unweighted": ("Rn[n] += W * (double)r2;", "Rn[n] += (double)r2;"),
    "cut-off comparison inverted": ("if (W > cuts->hi[n]) {", "if (W < cuts->hi[n]) {"),
    "cut-off survival probability q, not 1/q": ("if (!(u0 < 1.0 / cuts->q)) return ORC_LEAF_PRUNED;",
                                                "if (!(u0 < cuts->q)) return ORC_LEAF_PRUNED;"),
    "cut-off survivor not reweighted": ("Wp = W * cuts->q;", "Wp = W;"),
    "cut-offs applied at the empty walk": ("if (cuts && n > 0) {", "if (cuts) {"),
    "tour sums carried into the next tour": ("h->X[k] = 0.0;", "h->X[k] *= 1.0;"),
}


def _pins_hold(exact2):
    """A quick subset of tests/test_oracle_pins.py; False at the first failure."""
    # Philox known answer
    if list(orc.philox4x32_10([0, 0, 0, 0], [0, 0])) != [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]:
        return False
    # a_+ and free mask against an independent neighbour check
    for st in inputs.snapshot_batch(4, 2, 20, 60, n_lo=1):
        out = orc.step(2, 30, st["walk"], st["W"], st["Wsum"], st["M"], st["ordinal"],
                       st["seq"], st["tour"], seed=5)
        free = inputs.free_neighbours(st["walk"])
        if out["free_mask"] != sum(1 << j for j in free):
            return False
    # exact short lengths and first-tour chain
    h = orc.Oracle(2, 12, 3, seed=17)
    h.run(200)
    lc, S, rv = h.estimates()
    for n, c in enumerate([1, 4, 12, 36]):
        if not math.isclose(math.exp(lc[n]), c, rel_tol=1e-12):
            return False
    h1 = orc.Oracle(2, 20, 1, seed=3)
    h1.run(1)
    if h1.tables()["max_stack"] != 0:
        return False
    # probabilities of enrichment and survival (Sec. 2)
    walk = np.array([[0, 0], [1, 0], [1, 1]], dtype=np.int32)
    for target in (2.3, 0.37):
        M = 1 << 30
        Wsum = M / target - 1.0
        r = orc.ratio(2, 1.0, Wsum, M)
        hits = 0
        trials = 6000
        for k in range(trials):
            out = orc.step(2, 10, walk, 1.0, Wsum, M, k, 1, 2, seed=99)
            if target > 1:
                hits += out["c"] == 2
            else:
                hits += out["outcome"] == 3
        p = (math.ceil(r) - r) if target > 1 else r
        if abs(r - target) > 1e-6 or abs(hits / trials - p) > 5 * math.sqrt(p * (1 - p) / trials):
            return False
    # r = 1 at the empty walk whatever the table says (one child per tour)
    if orc.ratio(0, 3.0, 100.0, 7) != 1.0:
        return False
    # ordered pairs of distinct steps (c = 2 of three free steps) are uniform
    pairs = {}
    for k in range(6000):
        out = orc.step(2, 10, np.array([[0, 0], [1, 0]], dtype=np.int32), 1.0,
                       (1 << 29) - 1.0, 1 << 30, k, 0, 0, seed=11)
        pairs[tuple(out["dirs"])] = pairs.get(tuple(out["dirs"]), 0) + 1
    if len(pairs) != 6 or sum((v - 1000.0) ** 2 / 1000.0 for v in pairs.values()) > 5 + 6 * math.sqrt(10):
        return False
    # direction uniformity with c = 1 (three free steps)
    counts = np.zeros(4)
    for k in range(6000):
        out = orc.step(2, 10, np.array([[0, 0], [1, 0]], dtype=np.int32), 1.0,
                       (1 << 30) - 1.0, 1 << 30, k, 0, 0, seed=7)
        counts[out["dirs"][0]] += 1
    exp_ = 2000.0
    if counts[1] != 0 or sum((counts[[0, 2, 3]] - exp_) ** 2 / exp_) > 2 + 6 * 2:
        return False
    # counting theorem within 4 sigma, finite variance
    h = orc.Oracle(2, 12, 8, seed=1)
    h.run(1500)
    lc, S, rv = h.estimates()
    ex = np.array(exact2[:13], dtype=float)
    with np.errstate(divide="ignore", invalid="ignore"):
        z = (np.exp(lc - np.log(ex)) - 1.0) / np.sqrt(rv)
    zz = z[4:]
    if not (np.all(np.isfinite(zz)) and np.max(np.abs(zz)) < 4.0):
        return False
    # variance calibration, coarse: spread of z over seeds is O(1)
    zs = []
    for s in range(12):
        h = orc.Oracle(2, 10, 2, seed=500 + s)
        h.run(800)
        lc, S, rv = h.estimates()
        with np.errstate(divide="ignore", invalid="ignore"):
            zs.append((math.exp(lc[10] - math.log(exact2[10])) - 1.0) / math.sqrt(rv[10]))
    sd = float(np.std(zs))
    if not (0.4 < sd < 2.5):
        return False
    # original PERM with cut-offs (Sec. 2): no cut-off active is Rosenbluth, always
    # enriching grows a fixed tree, always pruning is binomial with exact reweighting
    h = orc.Oracle(2, 8, 2, seed=21)
    h.set_cutoffs(np.full(9, np.inf), np.zeros(9), 2, 2.0)
    h.run(300)
    t = h.tables()
    if t["max_stack"] != 0 or not np.all(t["S"][:7] == 600):
        return False
    h = orc.Oracle(2, 3, 1, seed=5)
    h.set_cutoffs(np.zeros(4), np.zeros(4), 3, 2.0)
    h.run(20)
    if list(h.tables()["S"]) != [20, 20, 60, 180]:
        return False
    lc, S, rv = h.estimates()
    if not (math.isclose(math.exp(lc[2]), 12.0, rel_tol=1e-12) and math.isclose(math.exp(lc[3]), 36.0, rel_tol=1e-12)):
        return False
    h = orc.Oracle(2, 3, 4, seed=77)
    h.set_cutoffs(np.full(4, np.inf), np.full(4, np.inf), 2, 3.0)
    h.run(2500)
    t = h.tables()
    p, M, S2 = 1.0 / 3.0, 10000, t["S"][2]
    if abs(S2 - M * p) > 5.0 * math.sqrt(M * p * (1 - p)):
        return False
    if not math.isclose(t["W"][2], S2 * 12.0 * 3.0 * 2.0 ** -orc.scale_exp(2, 2), rel_tol=1e-12):
        return False
    # per-tour square sums against the exact Rosenbluth second moment (no cut-off
    # active: one walk per tour, E[W^2] = sum over all walks of W)
    from tests.test_oracle_perm_cutoffs import _rosenbluth_moments
    count, e2, e4 = _rosenbluth_moments(2, 6)
    h = orc.Oracle(2, 6, 4, seed=61)
    h.set_cutoffs(np.full(7, np.inf), np.zeros(7), 2, 2.0)
    h.run(1000)
    t = h.tables()
    M = float(t["M"][0])
    for n in range(1, 7):
        s2 = (2.0 ** orc.scale_exp(2, n)) ** 2
        se = math.sqrt(max(e4[n] - e2[n] ** 2, 0.0) / M)
        if abs(t["Q"][n] * s2 / M - e2[n]) > 5.0 * se + 1e-9 * e2[n]:
            return False
    # the observable estimator (Sec. 1, eq. 5) against the exact mean |omega_n|^2
    c, r2 = orc.enumerate_r2(2, 10)
    h = orc.Oracle(2, 10, 6, seed=8)
    h.run(1500)
    est = h.mean_r2()
    if not np.all(np.abs(est[1:] / (r2[1:] / c[1:].astype(float)) - 1.0) < 0.03):
        return False
    return True


def _build_variant(src_text, tmpdir, name):
    c_path = os.path.join(tmpdir, name + ".c")
    so_path = os.path.join(tmpdir, name + ".so")
    with open(c_path, "w") as f:
        f.write(src_text)
    inc = os.path.dirname(SRC)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-I", inc, "-o", so_path, c_path, "-lm"], check=True)
    return so_path


def test_pins_detect_planted_mistakes():
    exact2 = load_counts(2)
    src = open(SRC).read()
    saved = orc._lib
    survivors = []
    try:
        with tempfile.TemporaryDirectory() as tmp:
            orc._lib = orc.configure(ctypes.CDLL(_build_variant(src, tmp, "orig")))
            assert _pins_hold(exact2), "pins must hold for the unmodified oracle"
            for i, (label, (old, new)) in enumerate(MUTATIONS.items()):
                assert src.count(old) == 1, label
                so = _build_variant(src.replace(old, new), tmp, "mut%d" % i)
                orc._lib = orc.configure(ctypes.CDLL(so))
                if _pins_hold(exact2):
                    survivors.append(label)
    finally:
        orc._lib = saved
    assert not survivors, "mistakes the pins did not catch: %s" % survivors
