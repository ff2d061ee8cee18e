"""Long walks: each walk's occupancy hash, site list and stack ring in the global
arena instead of shared memory (walk_memory = 2; the automatic choice for walks
too long for shared memory, n_max of 10^4).

- Rosenbluth chains of the original PERM with no cut-off active (Sec. 1; Sec. 2
  with T = inf, t = 0) are decided by the node alone, so a run is a deterministic
  function of the seed for any number of sequences: at n_max = 4096 on the cubic
  lattice (chains reach n_max, thousands of sites per walk) the GPU tables equal
  the oracle's (counts exactly, weights to 1e-12), with the walks in the arena
  and in shared memory alike.
- Interacting flatPERM sequences with the walks in the arena obey the counting
  theorem against exact c_n (Sec. 1, eq. 3)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from tests.gpu_util import Run, torch_cuda, zscores

pytestmark = pytest.mark.gpu

REL_W = 1e-12


def _close(a, b):
    return np.all(np.abs(a - b) <= REL_W * np.maximum(np.abs(a), np.abs(b)))


@pytest.mark.parametrize("d,n_max,N,tours,seed", [(3, 4096, 6, 8, 5), (2, 4096, 6, 40, 7)])
def test_long_rosenbluth_chains_equal_the_oracle(d, n_max, N, tours, seed):
    import paper_2002_03000_gb300 as pg
    torch_cuda()
    hi, lo = np.full(n_max + 1, np.inf), np.zeros(n_max + 1)
    o = orc.Oracle(d, n_max, N, seed)
    o.set_cutoffs(hi, lo, 2, 2.0)
    o.run(tours)
    ref = o.tables()
    got = {}
    for wm in (2, 1):
        with Run(d, n_max, N, seed, share_copies=-1, walk_memory=wm) as run:
            run.set_cutoffs(hi, lo, 2, 2.0)
            run.run(tours)
            got[wm] = run.tables()
            st = run.stats()
            assert st["status"] == 0 and st["steps"] == ref["steps"] and st["walk_memory"] == wm
        t = got[wm]
        assert np.array_equal(t["S"], ref["S"]), wm
        assert _close(t["W"], ref["W"]) and _close(t["Q"], ref["Q"]), wm
    if d == 3:
        assert ref["S"][n_max] > 0            # the chains reached n_max


@pytest.mark.parametrize("d,n_max,N,tours", [(2, 16, 300, 40), (3, 11, 300, 30)])
def test_arena_walks_obey_the_counting_theorem(d, n_max, N, tours, exact_counts):
    torch_cuda()
    with Run(d, n_max, N, 0xA12E4A + d, walk_memory=2) as run:
        run.run(tours)
        lc, S, rv = run.estimates()
        st = run.stats()
    M = N * tours
    assert st["status"] == 0
    assert S[0] == M and S[1] == M
    assert math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
    z = zscores(lc, rv, exact_counts[d][: n_max + 1])
    assert np.all(np.abs(z[2:]) < 4.5), z


def test_walks_too_long_for_shared_memory_use_the_arena():
    """n_max = 16000 on the square lattice: one walk's hash (2^15 slots) and site
    list need 160 KB beside the 128 KB snapshot table, more than a CTA's shared
    memory; the automatic choice puts the walks in the arena and runs.  Shared
    memory only is refused.  (At n_max = 10^4 one walk still fits beside its
    80 KB table.)"""
    import paper_2002_03000_gb300 as pg
    torch_cuda()
    with Run(2, 16000, 1, 1) as run:
        run.run(1)                               # the first tour: one chain (r = 1 at M = 1)
        st = run.stats()
        t = run.tables()
        assert st["status"] == 0 and st["steps"] == int(t["S"].sum()) and t["S"][0] == 1
        assert st["walk_memory"] == 2
        n_end = int(np.max(np.nonzero(t["S"])[0]))
        assert np.all(t["S"][: n_end + 1] == 1)
    with Run(2, 10000, 1, 1) as run:
        assert run.stats()["walk_memory"] == 1
    with pytest.raises(pg.PermError) as e:
        Run(2, 16000, 4, 1, walk_memory=1)
    assert e.value.code == pg._native.PERM_EUNSUPPORTED
