"""Original PERM with cut-offs (Sec. 2) on the GPU against the oracle.

With fixed cut-offs no decision reads the shared table, so a run whose tours
do not spread (fresh thresholds, or snapshot thresholds with sharing off) is
deterministic for any number of sequences: the GPU tables equal the oracle's
(sample counts exactly, weight sums and per-tour squares to relative 1e-12;
only the order of the sums differs).  Cut-offs are placed around the
asymptotic form of c_n (tests/inputs.py)."""
import math

import numpy as np
import pytest

import paper_2002_03000_gb300 as pg
from oracle import oracle as orc
from tests import inputs
from tests.gpu_util import REL_W, Run, torch_cuda, zscores

pytestmark = pytest.mark.gpu


def _cuts(d, n_max, f):
    return inputs.perm_cutoffs(d, n_max, f, lambda k: orc.scale_exp(d, k))


def _close(a, b):
    return np.all(np.abs(a - b) <= REL_W * np.maximum(np.abs(a), np.abs(b)))


# (d, n_max, sequences, tours, copies, q, f, algorithm, threshold, share_copies):
# many CTAs and ragged sequence counts; square and cubic; 64-bit keys (cubic n_max > 512)
CASES = [
    (2, 257, 300, 6, 2, 2.0, 1.5, pg.PERM_ALG2, pg.PERM_THRESH_FRESH, 0),
    (3, 200, 150, 6, 3, 3.0, 1.3, pg.PERM_ALG2, pg.PERM_THRESH_SNAPSHOT, -1),
    (2, 120, 37, 10, 2, 2.0, 1.3, pg.PERM_ALG1, pg.PERM_THRESH_FRESH, 0),
    (3, 700, 64, 3, 2, 2.0, 1.5, pg.PERM_ALG2, pg.PERM_THRESH_FRESH, 0),
    (2, 1000, 1000, 2, 4, 5.0, 1.5, pg.PERM_ALG2, pg.PERM_THRESH_SNAPSHOT, -1),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "d%d_n%d_N%d" % c[:3])
def test_whole_run_equals_oracle(case):
    torch_cuda()
    d, n_max, N, tours, copies, q, f, alg, thr, share = case
    hi, lo = _cuts(d, n_max, f)
    o = orc.Oracle(d, n_max, N, seed=41, alg=alg)
    o.set_cutoffs(hi, lo, copies, q)
    o.run(tours)
    t = o.tables()
    with Run(d, n_max, N, 41, alg=alg, threshold=thr, share_copies=share) as run:
        run.set_cutoffs(hi, lo, copies, q)
        run.run(tours)
        g = run.tables()
        st = run.stats()
    assert st["status"] == 0
    assert np.array_equal(g["M"], t["M"])
    assert np.array_equal(g["S"], t["S"])
    assert _close(g["W"], t["W"])
    assert _close(g["Q"], t["Q"])
    assert st["steps"] == t["steps"]


def test_cumulative_runs_and_switch_back_to_flatperm():
    """Cut-offs for the first tours, flatPERM after them: the same tables as the
    oracle doing the same (one sequence, fresh thresholds: deterministic)."""
    torch_cuda()
    d, n_max = 2, 90
    hi, lo = _cuts(d, n_max, 1.4)
    o = orc.Oracle(d, n_max, 1, seed=8)
    o.set_cutoffs(hi, lo, 3, 2.0)
    o.run(20)
    o.set_cutoffs(None, None)
    o.run(15)
    t = o.tables()
    with Run(d, n_max, 1, 8, threshold=pg.PERM_THRESH_FRESH) as run:
        run.set_cutoffs(hi, lo, 3, 2.0)
        run.run(20)
        run.set_cutoffs(None, None)
        run.run(15)
        g = run.tables()
    assert np.array_equal(g["S"], t["S"])
    assert _close(g["W"], t["W"])


def test_counting_theorem_with_shared_copies(exact_counts):
    """Snapshot thresholds with shared copies (the tours spread over walks, so
    the run is no longer deterministic): the estimates obey the counting theorem
    against exact c_n."""
    torch_cuda()
    for d, n_max, N in ((2, 16, 2000), (3, 11, 1500)):
        ex = exact_counts[d]
        hi = np.array([1.2 * ex[n] * 2.0 ** -orc.scale_exp(d, n) for n in range(n_max + 1)])
        lo = np.array([ex[n] / 1.2 * 2.0 ** -orc.scale_exp(d, n) for n in range(n_max + 1)])
        with Run(d, n_max, N, 5) as run:
            run.set_cutoffs(hi, lo, 2, 2.0)
            run.run(10)
            lc, S, rv = run.estimates()
            assert run.stats()["status"] == 0
        assert S[0] == N * 10
        z = zscores(lc, rv, ex[: n_max + 1])
        assert np.max(np.abs(z[2:])) < 5.0, z


def test_bad_cutoffs_are_rejected():
    torch_cuda()
    hi, lo = _cuts(2, 20, 1.5)
    with Run(2, 20, 4, 1) as run:
        for copies, q in ((0, 2.0), (5, 2.0), (2, 0.9)):
            with pytest.raises(pg.PermError):
                run.set_cutoffs(hi, lo, copies, q)
        with pytest.raises(ValueError):
            run.set_cutoffs(hi[:-1], lo[:-1], 2, 2.0)
