"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Holds none of the method's arithmetic: no weights, ratios, decisions or
random-number mapping -- only random self-avoiding walk snapshots (grown by
picking uniformly among unvisited neighbours and restarting when stuck) and
random scalar states in the ranges the method meets.
"""
import numpy as np

# unit steps in the order +x, -x, +y, -y, +z, -z
STEPS = {
    2: np.array([[1, 0], [-1, 0], [0, 1], [0, -1]], dtype=np.int64),
    3: np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                dtype=np.int64),
}


def random_saw(rng, d, n, max_restarts=100000):
    """A random n-step self-avoiding walk from the origin, shape (n+1, d)."""
    steps = STEPS[d]
    for _ in range(max_restarts):
        walk = [tuple([0] * d)]
        seen = {walk[0]}
        ok = True
        for _k in range(n):
            cur = np.array(walk[-1])
            cand = [tuple(cur + s) for s in steps]
            cand = [p for p in cand if p not in seen]
            if not cand:
                ok = False
                break
            p = cand[rng.integers(len(cand))]
            walk.append(p)
            seen.add(p)
        if ok:
            return np.array(walk, dtype=np.int32)
    raise RuntimeError("no walk found")


def free_neighbours(walk):
    """Directions (indices into STEPS) whose target site is not on the walk."""
    d = walk.shape[1]
    seen = {tuple(p) for p in walk.tolist()}
    end = walk[-1].astype(np.int64)
    return [j for j, s in enumerate(STEPS[d]) if tuple((end + s).tolist()) not in seen]


def random_state(rng, n):
    """Scalar state of a node: weight W, the sum Wsum of the weights recorded at
    its length before it, tours M, DFS ordinal, sequence and tour indices."""
    W = float(10.0 ** rng.uniform(-3, 3))
    M = int(rng.integers(1, 1 << 20))
    # Wsum is about M times a typical weight spread over three decades either
    # side of W (so the node's weight is sometimes above and sometimes below
    # the running average); sometimes exactly zero (first visit)
    Wsum = 0.0 if rng.random() < 0.05 else float(W * M * 10.0 ** rng.uniform(-1.5, 1.5))
    ordinal = int(rng.integers(0, 1 << 40))
    seq = int(rng.integers(0, 1 << 16))
    tour = int(rng.integers(0, 1 << 20))
    return dict(W=W, Wsum=Wsum, M=M, ordinal=ordinal, seq=seq, tour=tour)


def snapshot_batch(seed, d, n_max, count, n_lo=0):
    """count random snapshot states with walks of length in [n_lo, n_max]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_max + 1))
        walk = random_saw(rng, d, n)
        st = random_state(rng, n)
        st["walk"] = walk
        out.append(st)
    return out


def shortest_trapped_walk_2d(max_len=8):
    """A shortest square-lattice walk whose end-point has no free neighbour
    (iterative-deepening search), shape (n+1, 2)."""
    steps = STEPS[2]

    def search(walk, seen, depth):
        end = walk[-1]
        nbrs = [(end[0] + int(s[0]), end[1] + int(s[1])) for s in steps]
        if all(p in seen for p in nbrs):
            return list(walk)
        if depth == 0:
            return None
        for p in nbrs:
            if p not in seen:
                seen.add(p)
                walk.append(p)
                res = search(walk, seen, depth - 1)
                walk.pop()
                seen.discard(p)
                if res:
                    return res
        return None

    for limit in range(1, max_len + 1):
        res = search([(0, 0)], {(0, 0)}, limit)
        if res:
            return np.array(res, dtype=np.int32)
    return None


# growth constants and amplitude exponents of c_n ~ A mu^n n^(gamma - 1) from the
# literature (square: mu = 2.63815853, gamma = 43/32; cubic: mu = 4.6840386,
# gamma = 1.1570), used only to place cut-offs of the original PERM near c_n
_ASYMPTOTICS = {2: (2.63815853, 43.0 / 32.0, 1.18), 3: (4.6840386, 1.1570, 1.21)}


def perm_cutoffs(d, n_max, f, scale_exp):
    """Cut-offs T_n = f a_n and t_n = a_n / f around the asymptotic form a_n of
    c_n, at the stored weight scale 2^-scale_exp(n) (the scale function is passed
    in, so that this module holds none of the method's arithmetic)."""
    import math
    mu, gamma, amp = _ASYMPTOTICS[d]
    hi = np.empty(n_max + 1)
    lo = np.empty(n_max + 1)
    for n in range(n_max + 1):
        # in logs: mu^n alone leaves the double range at long lengths
        la = math.log(amp) + n * math.log(mu) + (gamma - 1.0) * math.log(max(n, 1)) - scale_exp(n) * math.log(2.0)
        hi[n] = f * math.exp(la)
        lo[n] = math.exp(la) / f
    return hi, lo
