"""Step parity: the CUDA growth step against the oracle on identical snapshot
states and random keys (through the C ABI).  Bit-exact for a_+, the free
mask, r (single precision), the enrichment count, the chosen steps and the
survival threshold; child weights to relative 1e-12."""
import numpy as np
import pytest

from oracle import oracle as orc
from tests import inputs
from tests.gpu_util import debug_philox, debug_step

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


def _compare(states, d, n_max, seed):
    oi, r, w, K = debug_step(states, d, n_max, seed)
    mism = []
    for b, st in enumerate(states):
        ref = orc.step(d, n_max, st["walk"], st["W"], st["T"], st["M"], st["ordinal"],
                       st["seq"], st["tour"], seed)
        got = dict(outcome=int(oi[b, 0]), a_plus=int(oi[b, 1]), free_mask=int(oi[b, 2]),
                   c=int(oi[b, 3]), dirs=[int(x) for x in oi[b, 4:4 + max(int(oi[b, 3]), 0)]])
        ok = (got["outcome"] == ref["outcome"] and got["a_plus"] == ref["a_plus"] and
              got["free_mask"] == ref["free_mask"] and got["c"] == ref["c"] and
              got["dirs"] == ref["dirs"])
        if ref["outcome"] >= 2:
            ok &= np.float32(r[b]).tobytes() == np.float32(ref["r"]).tobytes()
            ok &= int(K[b]) == int(ref["survive_K"])
        if ref["outcome"] == 3:
            ok &= abs(w[b] - ref["child_w"]) <= REL_W * abs(ref["child_w"])
        if not ok:
            mism.append((b, got, ref, float(r[b]), float(w[b]), int(K[b])))
    assert not mism, mism[:3]


@pytest.mark.parametrize("d,n_max", [(2, 40), (2, 512), (3, 30), (3, 512)])
def test_step_parity_random_states(d, n_max):
    states = inputs.snapshot_batch(100 + d * 7 + n_max, d, min(n_max, 200), 1500)
    _compare(states, d, n_max, seed=0x1234ABCD5678EF01)


@pytest.mark.parametrize("d", [2, 3])
def test_step_parity_edge_cases(d):
    rng = np.random.default_rng(9)
    n_max = 24
    states = []
    # the empty walk, with and without table data
    for T in (0.0, 3.0, 1e9):
        states.append(dict(walk=np.zeros((1, d), dtype=np.int32), W=1.0, T=T, M=7, ordinal=0,
                           seq=1, tour=2))
    # walks at n_max (leaf), first visits (T = 0), r exactly 1 and 2 (p = 0)
    for k in range(60):
        n = n_max if k % 3 == 0 else int(rng.integers(1, n_max))
        w = inputs.random_saw(rng, d, n)
        M = 1 << 30
        T = [0.0, 1.0 - 1.0 / M, 0.5 - 1.0 / M, 1e-30, 1e30][k % 5]
        states.append(dict(walk=w, W=1.0, T=T, M=M, ordinal=int(rng.integers(0, 1 << 40)),
                           seq=k, tour=3 * k))
    # a trapped walk (d = 2): the end-point has no free neighbour
    if d == 2:
        trapped = inputs.shortest_trapped_walk_2d()
        states.append(dict(walk=trapped, W=2.0, T=1.0, M=10, ordinal=5, seq=0, tour=0))
    # huge and tiny M, big ordinals
    for M in (1, 2, (1 << 62)):
        w = inputs.random_saw(rng, d, 5)
        states.append(dict(walk=w, W=3.5, T=1.25, M=M, ordinal=(1 << 63) + 12345, seq=2 ** 31,
                           tour=2 ** 32 - 1))
    _compare(states, d, n_max, seed=42)


def test_step_parity_many_keys():
    """Same state, many counters: the decision and the chosen steps follow the key."""
    walk = np.array([[0, 0], [1, 0], [1, 1]], dtype=np.int32)
    states = [dict(walk=walk, W=1.0, T=1.0 / 2.3 - 1.0 / (1 << 30), M=1 << 30, ordinal=k,
                   seq=7, tour=11) for k in range(3000)]
    _compare(states, 2, 10, seed=99)
    states = [dict(walk=walk, W=1.0, T=1.0 / 0.37 - 1.0 / (1 << 30), M=1 << 30, ordinal=k,
                   seq=7, tour=11) for k in range(3000)]
    _compare(states, 2, 10, seed=99)
