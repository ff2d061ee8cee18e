"""Copies grown on other walks ("shared copies").

Sec. 2 grows the c copies of an enriched state independently of each other,
so a waiting copy may be grown by any walk.  A walk with no tour to start
(the admission limit early in a run, or no tickets left at its end) takes the
oldest waiting copy of another walk's tour, rebuilds the walk up to the branch
point and grows the copy's subtree; the weights of that part still count for
the tour that made the copy (its per-tour sum, and the tour finishes once
all of its parts have).  The runs here start with most walks idle, so many
copies move: every tour still finishes exactly once, the estimates stay
unbiased (c_n within 4.5 sigma of the exact counts, S_0 = S_1 = M), and sampled
nodes of moved parts (ordinal high word = part id) replay bit for bit in the
oracle's growth step.
"""
import math

import numpy as np
import pytest

from tests.gpu_util import Run, replay, torch_cuda, zscores

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,n_max,N,tours,every", [(2, 200, 64, 64, 7), (3, 120, 64, 64, 5)])
def test_moved_parts_replay_and_estimates(d, n_max, N, tours, every, exact_counts):
    torch_cuda()
    seed = 3
    cap = 4000
    with Run(d, n_max, N, seed) as run:
        run.trace_enable(every, 1, cap)
        run.run(tours)
        count, recs, coords = run.trace_read()
        lc, S, rv = run.estimates()
        st = run.stats()
        M = run.tables()["M"][0]
    assert st["status"] == 0
    assert st["shared"] > 0
    assert M == N * tours and st["tours_finished"] == M
    assert S[0] == M and S[1] == M
    assert math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
    moved = sum(1 for r in recs if int(r.ordinal) >> 32)
    assert moved > 20, (moved, len(recs))
    bad = replay(recs, coords, d, n_max, seed)
    assert not bad, bad[:3]
    ex = exact_counts[d]
    z = zscores(lc, rv, ex[: min(len(ex), n_max + 1)])
    assert np.all(np.abs(z[2:]) < 4.5), z


def test_sharing_off_moves_nothing():
    torch_cuda()
    with Run(2, 200, 64, 3, share_copies=-1) as run:
        run.run(16)
        st = run.stats()
    assert st["status"] == 0 and st["shared"] == 0 and st["tours_finished"] == 64 * 16


def test_cumulative_runs_with_sharing():
    """Repeated launches continue the same run; every launch ends with all of
    its tours finished and no copy left in the ring."""
    torch_cuda()
    with Run(2, 300, 128, 5) as run:
        for k in range(1, 4):
            run.run(8)
            st = run.stats()
            assert st["status"] == 0
            assert st["tours_finished"] == 128 * 8 * k
        lc, S, rv = run.estimates()
    assert S[0] == 128 * 24 and math.isclose(math.exp(lc[1]), 4.0, rel_tol=1e-12)


@pytest.mark.parametrize("d,n_max,N,tours", [(3, 945, 2142, 4), (2, 1725, 422, 4)])
def test_startup_trees_finish(d, n_max, N, tours):
    """Start-up trees that one walk cannot grow in minutes (square lattice,
    n_max 1725), and a run where unbounded spreading of parts runs away (cubic,
    n_max 945): both finish in seconds with the default cap and its stall boost."""
    import time
    torch_cuda()
    with Run(d, n_max, N, 1, max_seconds=60.0) as run:
        t0 = time.perf_counter()
        run.run(tours)
        el = time.perf_counter() - t0
        st = run.stats()
        lc, S, rv = run.estimates()
    assert st["status"] == 0 and st["tours_finished"] == N * tours
    assert el < 20.0, el
    assert S[0] == N * tours and math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
    assert np.all(S > 0)


def test_share_cap_argument():
    import paper_2002_03000_gb300 as pg
    torch_cuda()
    with Run(2, 100, 64, 1, share_copies=2) as run:
        run.run(8)
        assert run.stats()["status"] == 0
    for bad in (-2, 2000):
        with pytest.raises(pg.PermError):
            Run(2, 100, 64, 1, share_copies=bad)


@pytest.mark.parametrize("d,n_max,N,helpers,tours", [(2, 200, 12, 300, 200), (3, 120, 12, 300, 200)])
def test_helper_walks(d, n_max, N, helpers, tours, exact_counts):
    """Walks beyond one per sequence start no tour and grow waiting copies only:
    the tours are the sequences' own (M = N x tours, each finishing once), copies
    move to the helpers, and the estimates meet exact c_n within 4.5 sigma; sampled
    nodes of moved parts replay bit for bit in the oracle."""
    torch_cuda()
    seed = 17
    with Run(d, n_max, N, seed, helper_walks=helpers) as run:
        run.trace_enable(5, 1, 3000)
        run.run(tours)
        lc, S, rv = run.estimates()
        st = run.stats()
        count, recs, coords = run.trace_read()
    M = N * tours
    assert st["status"] == 0 and st["slots"] > N
    assert st["tours"] == M and st["tours_finished"] == M and st["shared"] > 0
    assert S[0] == M and S[1] == M
    assert math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
    top = 16 if d == 2 else 11
    z = zscores(lc, rv, exact_counts[d][: top + 1])
    assert np.all(np.abs(z[2:]) < 4.5), z
    moved = [rec for rec in recs if (rec.ordinal >> 32) != 0]
    assert moved
    assert not replay(recs, coords, d, n_max, seed)


def test_helper_walks_need_shared_copies():
    import paper_2002_03000_gb300 as pg
    torch_cuda()
    for kw in (dict(share_copies=-1), dict(threshold=pg.PERM_THRESH_FRESH), dict(alg=pg.PERM_ALG1)):
        with pytest.raises(pg.PermError):
            Run(2, 32, 4, 1, helper_walks=8, **kw)
        with Run(2, 32, 4, 1, **kw) as run:          # the default adds none there
            assert run.stats()["slots"] == 4
    with Run(2, 32, 4, 1, helper_walks=0) as run:
        assert run.stats()["slots"] == 4
    with Run(2, 32, 4, 1) as run:                    # default: none
        assert run.stats()["slots"] == 4
    with Run(2, 32, 4, 1, helper_walks=-1) as run:   # -1: the layout's spare walks
        assert run.stats()["slots"] > 4


def test_helper_walks_default_none_and_fill_option():
    """No helper walks unless asked; helper_walks = -1 fills the automatic layout's
    room beyond the tour walks, and every tour still finishes once."""
    torch_cuda()
    with Run(2, 64, 12, 3) as run:
        run.run(4)
        plain = run.stats()
    with Run(2, 64, 12, 3, helper_walks=-1) as run:
        run.run(4)
        filled = run.stats()
    assert plain["status"] == 0 and filled["status"] == 0
    assert plain["slots"] == 12 and filled["slots"] > 12
    assert plain["tours_finished"] == filled["tours_finished"] == 48
