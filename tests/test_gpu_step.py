"""Step parity: the CUDA growth step against the oracle on identical snapshot
states and random keys (through the C ABI).  Bit-exact for a_+, the free
mask, the enrichment count or survival, and the chosen steps; r bit for bit
where the kernel evaluated it in double precision, else within its estimate's
bound; child weights to relative 1e-12.  Both the kernel's own path and the
path that evaluates every r in double precision are checked, and states placed
next to every decision boundary make the kernel fall back to the exact r."""
import numpy as np
import pytest

from oracle import oracle as orc
from tests import inputs
from tests.gpu_util import debug_philox, debug_step, same_step

pytestmark = pytest.mark.gpu

REL_W = 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_philox_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    ctrs = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctrs[0] = 0
    ctrs[1] = 0xFFFFFFFF
    key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
    got = debug_philox(ctrs, key)
    for b in range(ctrs.shape[0]):
        assert list(got[b]) == list(orc.philox4x32_10(ctrs[b], key)), b


def _compare(states, d, n_max, seed, force_exact=0):
    oi, r, w = debug_step(states, d, n_max, seed, force_exact=force_exact)
    mism = []
    for b, st in enumerate(states):
        ref = orc.step(d, n_max, st["walk"], st["W"], st["Wsum"], st["M"], st["ordinal"],
                       st["seq"], st["tour"], seed)
        c = int(oi[b, 3])
        got = dict(outcome=int(oi[b, 0]), a_plus=int(oi[b, 1]), free_mask=int(oi[b, 2]),
                   c=c, dirs=[int(x) for x in oi[b, 4:4 + max(c, 0)]], exact=int(oi[b, 10]),
                   r=float(r[b]), child_w=float(w[b]))
        if force_exact and ref["outcome"] >= 2 and st["walk"].shape[0] > 1:
            assert got["exact"] == 1          # (the empty walk has r = 1 by definition)
        if not same_step(got, ref):
            mism.append((b, got, ref))
    assert not mism, mism[:3]
    return oi[:, 10]


@pytest.mark.parametrize("d,n_max", [(2, 40), (2, 512), (3, 30), (3, 512)])
@pytest.mark.parametrize("force_exact", [0, 1])
def test_step_parity_random_states(d, n_max, force_exact):
    states = inputs.snapshot_batch(100 + d * 7 + n_max, d, min(n_max, 200), 1500)
    _compare(states, d, n_max, seed=0x1234ABCD5678EF01, force_exact=force_exact)


@pytest.mark.parametrize("d", [2, 3])
def test_step_parity_edge_cases(d):
    rng = np.random.default_rng(9)
    n_max = 24
    states = []
    # the empty walk, with and without table data
    for Wsum in (0.0, 3.0, 1e9):
        states.append(dict(walk=np.zeros((1, d), dtype=np.int32), W=1.0, Wsum=Wsum, M=7, ordinal=0,
                           seq=1, tour=2))
    # walks at n_max (leaf), first visits (Wsum = 0), r exactly 1 and 2 (p = 0), and
    # ratios beyond the estimate's range (Wsum/W of 2^-1000 and 2^1000)
    for k in range(70):
        n = n_max if k % 3 == 0 else int(rng.integers(1, n_max))
        w = inputs.random_saw(rng, d, n)
        M = 1 << 30
        Wsum = [0.0, M - 1.0, M / 2 - 1.0, 1e-30, 1e30, 2.0 ** -1000, 2.0 ** 1000][k % 7]
        states.append(dict(walk=w, W=1.0, Wsum=Wsum, M=M, ordinal=int(rng.integers(0, 1 << 40)),
                           seq=k, tour=3 * k))
    # a trapped walk (d = 2): the end-point has no free neighbour
    if d == 2:
        trapped = inputs.shortest_trapped_walk_2d()
        states.append(dict(walk=trapped, W=2.0, Wsum=1.0, M=10, ordinal=5, seq=0, tour=0))
    # huge and tiny M, big ordinals
    for M in (1, 2, (1 << 62)):
        w = inputs.random_saw(rng, d, 5)
        states.append(dict(walk=w, W=3.5, Wsum=1.25 * M, M=M, ordinal=(1 << 63) + 12345, seq=2 ** 31,
                           tour=2 ** 32 - 1))
    # first tour: the node's own weight is the whole sum, r = 1 exactly
    for k in range(10):
        w = inputs.random_saw(rng, d, int(rng.integers(1, n_max)))
        states.append(dict(walk=w, W=float(10.0 ** rng.uniform(-5, 5)), Wsum=0.0, M=1,
                           ordinal=int(rng.integers(0, 1 << 40)), seq=k, tour=0))
    for fe in (0, 1):
        _compare(states, d, n_max, seed=42, force_exact=fe)


def test_step_parity_many_keys():
    """Same state, many counters: the decision and the chosen steps follow the key."""
    walk = np.array([[0, 0], [1, 0], [1, 1]], dtype=np.int32)
    M = 1 << 30
    for target in (2.3, 0.37):
        states = [dict(walk=walk, W=1.0, Wsum=M / target - 1.0, M=M, ordinal=k,
                       seq=7, tour=11) for k in range(3000)]
        _compare(states, 2, 10, seed=99)


def _boundary_states(rng, d, n_max, seed, count):
    """States whose r lies within a few units in the last place of a decision
    boundary for the node's own first random word: u0 + r = ceil(r) (enrichment,
    c = floor or ceil), r = u0 (survival), r = 1 (the branch) and r = an integer.
    The word comes from the oracle's Philox for the node's counter; Wsum is
    chosen so that W M / (Wsum + W) lands on the boundary (W = 1)."""
    states = []
    for k in range(count):
        n = int(rng.integers(1, min(n_max, 40)))
        walk = inputs.random_saw(rng, d, n)
        ordinal, sq, tr = int(rng.integers(0, 1 << 40)), int(rng.integers(0, 1 << 16)), k
        w0 = int(orc.philox4x32_10([ordinal & 0xFFFFFFFF, ordinal >> 32, tr, sq],
                                   [seed & 0xFFFFFFFF, seed >> 32])[0])
        u0 = w0 / 2.0 ** 32
        kind = k % 4
        if kind == 0:
            target = 2.0 - u0                                    # u0 = ceil(r) - r
        elif kind == 1:
            target = u0 if u0 > 1e-6 else 0.5                    # u0 = r
        elif kind == 2:
            target = 1.0                                         # the branch
        else:
            target = 2.0                                         # floor r = ceil r
        M = int(rng.integers(1 << 20, 1 << 40))
        base = M / target - 1.0
        # a few ulp either side of the boundary
        Wsum = float(np.nextafter(base, np.inf * int(rng.choice([-1, 1])))) if base > 0 else 0.0
        for _ in range(int(rng.integers(0, 4))):
            Wsum = float(np.nextafter(Wsum, np.inf if rng.random() < 0.5 else -np.inf))
        states.append(dict(walk=walk, W=1.0, Wsum=max(Wsum, 0.0), M=M, ordinal=ordinal, seq=sq, tour=tr))
    return states


@pytest.mark.parametrize("d", [2, 3])
def test_step_parity_at_decision_boundaries(d):
    """Nodes placed on the decision boundaries: the estimate cannot settle them,
    the kernel falls back to the exact r, and the decisions equal the oracle's."""
    seed = 0x0DDBA11
    rng = np.random.default_rng(20 + d)
    states = _boundary_states(rng, d, 64, seed, 2000)
    exact = _compare(states, d, 64, seed)
    assert np.mean(exact) > 0.9, np.mean(exact)


def test_step_exact_fallback_is_rare_on_random_states():
    """On states spread like a run's (first visits left out: there r is within an
    ulp of the integer M by definition), few nodes need the exact r."""
    states = [s for s in inputs.snapshot_batch(77, 2, 100, 4000) if s["Wsum"] > 0.0]
    exact = _compare(states, 2, 100, seed=5)
    assert np.mean(exact) < 1e-3, np.mean(exact)
