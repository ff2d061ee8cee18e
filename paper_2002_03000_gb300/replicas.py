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


def estimates(tables: dict, d: int):
    """(log c_n, S_n, relative variance of c_n) from raw Algorithm-2 tables,
    pooled or not, by the library's perm_estimates_from_tables (eq. 4 on the
    pooled sums: c_n = W_n / M, var = (Q_n / M - c_n^2) / (M - 1))."""
    from . import _native
    W = np.asarray(tables["W"], dtype=np.float64)
    S = np.asarray(tables["S"], dtype=np.float64)
    M = np.asarray(tables["M"], dtype=np.int64).reshape(-1)
    L = W.size
    if M.size != 1:
        raise ValueError("estimates take Algorithm-2 tables (one row)")
    if M[0] < 1:
        return np.full(L, -math.inf), S.copy(), np.full(L, math.inf)
    lc, rv = _native.perm_estimates_from_tables(d, L - 1, W, tables["Q"], M)
    return lc, S.copy(), rv
