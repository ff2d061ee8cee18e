"""Checkpoint and resume at a tour boundary: a run saved, loaded into a new
handle and continued equals the run grown without interruption, where the
run is deterministic (sharing off); for interacting runs the tour counters
continue and the estimates obey the counting theorem."""
import math

import numpy as np
import pytest

import paper_2002_03000_gb300 as pg
from oracle import oracle as orc
from tests import inputs
from tests.gpu_util import REL_W, Run, torch_cuda, zscores

pytestmark = pytest.mark.gpu


def _close(a, b):
    return np.all(np.abs(a - b) <= REL_W * np.maximum(np.abs(a), np.abs(b)))


@pytest.mark.parametrize("d,n_max,N,alg,first,rest", [
    (2, 64, 1, pg.PERM_ALG2, 30, 20),
    (3, 40, 24, pg.PERM_ALG1, 6, 5),
])
def test_resume_equals_uninterrupted(tmp_path, d, n_max, N, alg, first, rest):
    torch_cuda()
    path = str(tmp_path / "run.ckpt")
    with Run(d, n_max, N, 13, alg=alg, threshold=pg.PERM_THRESH_FRESH, observables=1) as a:
        a.run(first + rest)
        ta = a.tables()
        ra = a.mean_r2()[1]
        sa = a.stats()
    with Run(d, n_max, N, 13, alg=alg, threshold=pg.PERM_THRESH_FRESH, observables=1) as b:
        b.run(first)
        b.save(path)
    c = pg.Run.load(path)
    try:
        assert (c.d, c.n_max, c.n_seq, c.alg) == (d, n_max, N, alg)
        c.run(rest)
        tc = c.tables()
        rc = c.mean_r2()[1]
        sc = c.stats()
    finally:
        c.close()
    assert np.array_equal(tc["M"], ta["M"])
    assert np.array_equal(tc["S"], ta["S"])
    assert _close(tc["W"], ta["W"]) and _close(tc["Q"], ta["Q"]) and _close(rc, ra)
    assert sc["steps"] == sa["steps"] and sc["status"] == 0


def test_resume_with_cutoffs_equals_the_oracle(tmp_path):
    """Original PERM with many sequences (deterministic with sharing off): the
    cut-offs travel in the checkpoint, and the resumed run equals the oracle."""
    torch_cuda()
    d, n_max, N = 2, 200, 64
    hi, lo = inputs.perm_cutoffs(d, n_max, 1.5, lambda k: orc.scale_exp(d, k))
    o = orc.Oracle(d, n_max, N, seed=5)
    o.set_cutoffs(hi, lo, 2, 2.0)
    o.run(7)
    t = o.tables()
    path = str(tmp_path / "cut.ckpt")
    with Run(d, n_max, N, 5, share_copies=-1) as b:
        b.set_cutoffs(hi, lo, 2, 2.0)
        b.run(4)
        b.save(path)
    with pg.Run.load(path) as c:
        c.run(3)
        g = c.tables()
    assert np.array_equal(g["S"], t["S"]) and np.array_equal(g["M"], t["M"])
    assert _close(g["W"], t["W"])


def test_interacting_run_resumes(tmp_path, exact_counts):
    torch_cuda()
    path = str(tmp_path / "snap.ckpt")
    with Run(2, 16, 2000, 3) as b:
        b.run(5)
        b.save(path)
    with pg.Run.load(path) as c:
        c.run(5)
        lc, S, rv = c.estimates()
        st = c.stats()
        M = c.tables()["M"][0]
    assert st["status"] == 0 and M == 2000 * 10 and S[0] == M
    assert st["tours_finished"] == M
    z = zscores(lc, rv, exact_counts[2][:17])
    assert np.max(np.abs(z[2:])) < 4.5, z
