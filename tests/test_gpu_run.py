"""Whole-run parity of the persistent CUDA kernel against the oracle.

- fresh thresholds with one sequence, and Algorithm 1 with many sequences:
  every node sees exactly the table the sequential oracle sees, so the tables
  agree node for node (counts exactly, weights to relative 1e-12);
- snapshot thresholds (the benchmarked form of Algorithm 2): estimates agree
  with exact c_n and with the oracle within 4 standard errors, c_0 and c_1
  are exact, and sampled nodes of full-size runs replay bit for bit in the
  oracle's growth step.
"""
import math

import numpy as np
import pytest

import paper_2002_03000_gb300 as pg
from oracle import oracle as orc
from tests.gpu_util import REL_W, SIGMA_FLOOR, Run, replay, torch_cuda, zscores

pytestmark = pytest.mark.gpu



def _rel_close(a, b, rel):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    return np.all(np.abs(a - b) <= rel * np.maximum(np.abs(a), np.abs(b)))


@pytest.mark.parametrize("d,n_max,tours", [(2, 16, 3000), (2, 100, 300), (3, 20, 1000), (3, 600, 40)])
def test_fresh_single_sequence_matches_oracle(d, n_max, tours):
    torch_cuda()
    seed = 0xC0FFEE + d
    with Run(d, n_max, 1, seed, threshold=pg.PERM_THRESH_FRESH) as run:
        run.run(tours // 2)
        run.run(tours - tours // 2)            # cumulative calls continue the run
        g = run.tables()
        st = run.stats()
    o = orc.Oracle(d, n_max, 1, seed)
    o.run(tours)
    t = o.tables()
    assert st["status"] == 0
    assert g["M"][0] == t["M"][0] == tours
    assert np.array_equal(g["S"], t["S"])
    assert _rel_close(g["W"], t["W"], REL_W)
    assert _rel_close(g["Q"], t["Q"], REL_W)
    assert st["steps"] == t["steps"]


@pytest.mark.parametrize("d,n_max,N,tours", [(2, 30, 300, 40), (3, 24, 200, 30)])
def test_alg1_matches_oracle(d, n_max, N, tours):
    """Algorithm 1: every sequence has its own table; each row is sequential
    flatPERM and must match the oracle's row."""
    torch_cuda()
    seed = 777
    with Run(d, n_max, N, seed, alg=pg.PERM_ALG1) as run:
        run.run(tours)
        g = run.tables()
        lc_g, S_g, rv_g = run.estimates()
    o = orc.Oracle(d, n_max, N, seed, alg=orc.ORC_ALG1)
    o.run(tours)
    t = o.tables()
    lc_o, S_o, rv_o = o.estimates()
    assert np.array_equal(g["M"], t["M"])
    assert np.array_equal(g["S"], t["S"])
    assert _rel_close(g["W"], t["W"], REL_W)
    assert _rel_close(g["Q"], t["Q"], REL_W)
    assert np.allclose(lc_g, lc_o, rtol=0, atol=1e-10)


@pytest.mark.parametrize("d,n_max,N,tours", [(2, 16, 12, 20000), (3, 11, 12, 8000), (2, 16, 4096, 40)])
def test_snapshot_counting_theorem(d, n_max, N, tours, exact_counts):
    """Snapshot thresholds keep the estimator unbiased: c_n within 4.5 sigma of the
    exact counts at every length (shared thresholds correlate the tours, so the
    per-tour variance slightly understates the spread); c_0 = 1 and c_1 = 2d
    exactly; S_0 = S_1 = M."""
    torch_cuda()
    with Run(d, n_max, N, seed=1) as run:
        run.run(tours)
        lc, S, rv = run.estimates()
        st = run.stats()
        M = run.tables()["M"][0]
    assert st["status"] == 0
    assert M == N * tours
    assert S[0] == M and S[1] == M
    assert math.isclose(math.exp(lc[0]), 1.0, rel_tol=1e-12)
    assert math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
    z = zscores(lc, rv, exact_counts[d][: n_max + 1])
    assert np.all(np.isfinite(z[2:])) and np.max(np.abs(z[2:])) < 4.5, z
    # and against the oracle (independent runs): combined 4.5 sigma
    o = orc.Oracle(d, n_max, N, seed=2)
    o.run(min(tours, max(1, 200000 // N)))
    lo, So, rvo = o.estimates()
    diff = lc[2:] - lo[2:]
    var = rv[2:] + rvo[2:] + 2 * SIGMA_FLOOR ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        zz = np.where((np.abs(diff) < 1e-12) & (var == 0.0), 0.0, diff / np.sqrt(var))
    assert np.all(np.abs(zz) < 4.5), zz


@pytest.mark.parametrize("d,n_max,N,tours,every,tour_every",
                         [(2, 512, 4096, 256, 97, 53), (3, 512, 8192, 128, 89, 41)])
def test_full_size_sampled_nodes_replay(d, n_max, N, tours, every, tour_every, exact_counts):
    """Full-size runs in the benchmarked launch form: sampled nodes (with the
    walk, weight, threshold and tour count they saw) replay bit for bit in the
    oracle's growth step; properties that hold at any size hold."""
    torch_cuda()
    seed = 1
    cap = 3000
    with Run(d, n_max, N, seed) as run:
        run.trace_enable(every, tour_every, cap)
        run.run(tours)
        count, recs, coords = run.trace_read()
        lc, S, rv = run.estimates()
        st = run.stats()
        M = run.tables()["M"][0]
    assert st["status"] == 0
    assert count > 200
    bad = replay(recs, coords, d, n_max, seed)
    assert not bad, bad[:3]
    assert M == N * tours and S[0] == M and S[1] == M
    assert math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
    ex = exact_counts[d]
    z = zscores(lc, rv, ex[: min(len(ex), n_max + 1)])
    assert np.all(np.abs(z[2:]) < 4.5), z
    # every length up to n_max is reached, and the histogram is roughly flat
    assert np.all(S > 0)
    assert 0.2 < S[n_max] / M < 5.0


def test_bad_arguments_rejected():
    torch_cuda()
    for args in [(1, 10, 4), (4, 10, 4), (2, 0, 4), (2, 10, 0)]:
        with pytest.raises(pg.PermError):
            Run(*args, seed=1)
    with pytest.raises(pg.PermError):
        Run(3, 5000000, 4, seed=1)
