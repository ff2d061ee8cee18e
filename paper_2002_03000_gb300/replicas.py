"""Replicas on several GPUs: one process per GPU, each growing an independent
Algorithm-2 run (its own run id, hence its own random streams), pooled on the
host.

There is no exchange step on the growth path: the replicas' tours are
independent, so their raw tables add up to the tables of one run of all their
tours with independent thresholds per replica.  Pooled, the sample average of
Sec. 1, eq. 4 is sum W_n / sum M, an unbiased estimate of c_n, and its variance
follows from the summed per-tour squares Q_n as for a single run.  Timing over
the replicas is the slowest replica's time (all run at once) against the sum of
their growth steps.

Collectives go through torch.distributed (NCCL between GPUs; gloo on the host
for tests).  With no process group, or one process, every function is the
identity."""
from __future__ import annotations

import math

import numpy as np


def _group():
    try:
        import torch.distributed as dist
    except ImportError:
        return None
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return None
    return dist


def reduce_timing(seconds: float, steps: float, device=None):
    """(max of seconds, sum of steps) over the process group."""
    dist = _group()
    if dist is None:
        return float(seconds), float(steps)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    s = torch.tensor([float(steps)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), float(s.item())


def pool_tables(tables: dict, device=None) -> dict:
    """Sum of the raw Algorithm-2 tables (W_n, S_n, Q_n at the stored scale, M)
    over the process group; the input dict is the one Run.tables() returns."""
    dist = _group()
    W = np.asarray(tables["W"], dtype=np.float64)
    S = np.asarray(tables["S"], dtype=np.float64)
    Q = np.asarray(tables["Q"], dtype=np.float64)
    M = np.asarray(tables["M"], dtype=np.int64)
    if M.size != 1:
        raise ValueError("pooling takes Algorithm-2 tables (one row)")
    if dist is None:
        return dict(W=W.copy(), S=S.copy(), Q=Q.copy(), M=M.copy())
    import torch
    L = W.size
    flat = torch.tensor(np.concatenate([W, S, Q]), dtype=torch.float64, device=device)
    m = torch.tensor(M, dtype=torch.int64, device=device)
    dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.SUM)
    f = flat.cpu().numpy()
    return dict(W=f[:L].copy(), S=f[L:2 * L].copy(), Q=f[2 * L:].copy(), M=m.cpu().numpy())


def scale_exp(d: int, n: int) -> int:
    """Exponent of the stored weight scale (stored = W / 2^E(n)), as the library
    stores it: floor(11 n / 8) on the square lattice, floor(9 n / 4) on the cubic."""
    return (11 * n) // 8 if d == 2 else (9 * n) // 4


def estimates(tables: dict, d: int):
    """(log c_n, S_n, relative variance of c_n) from raw Algorithm-2 tables,
    pooled or not: c_n = W_n / M (eq. 4), var = (Q_n / M - c_n^2) / (M - 1)."""
    W, S, Q = (np.asarray(tables[k], dtype=np.float64) for k in ("W", "S", "Q"))
    M = int(np.asarray(tables["M"]).reshape(-1)[0])
    L = W.size
    lc = np.full(L, -math.inf)
    rv = np.full(L, math.inf)
    if M >= 1:
        c = W / float(M)
        pos = c > 0.0
        lc[pos] = np.log(c[pos]) + np.array([scale_exp(d, n) for n in range(L)])[pos] * math.log(2.0)
        if M >= 2:
            var = np.maximum((Q / float(M) - c * c) / float(M - 1), 0.0)
            rv[pos] = var[pos] / (c[pos] * c[pos])
    return lc, S.copy(), rv
