"""Replicas pooled across processes (the multi-GPU form, one process per GPU),
exercised on the host: two gloo ranks, each with the tables of an independent
oracle run, pool them and reduce their timing."""
import math
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2002_03000_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_tables(seed, d=2, n_max=12, n_seq=4, tours=300):
    h = orc.Oracle(d, n_max, n_seq, seed=seed)
    h.run(tours)
    t = h.tables()
    return dict(W=t["W"], S=t["S"], Q=t["Q"], M=t["M"])


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pooled = replicas.pool_tables(_oracle_tables(100 + rank))
        sec, steps = replicas.reduce_timing(1.5 * (rank + 1), 10.0 * (rank + 1))
        out.put((rank, pooled, sec, steps))
    finally:
        dist.destroy_process_group()


def test_two_ranks_pool_tables_and_timing(exact_counts):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = _oracle_tables(100), _oracle_tables(101)
    for rank, pooled, sec, steps in res:
        # every rank holds the sum of both runs' raw tables
        assert np.array_equal(pooled["S"], a["S"] + b["S"])
        assert np.allclose(pooled["W"], a["W"] + b["W"], rtol=1e-15, atol=0)
        assert np.allclose(pooled["Q"], a["Q"] + b["Q"], rtol=1e-15, atol=0)
        assert int(pooled["M"][0]) == int(a["M"][0] + b["M"][0])
        # the slowest replica's time, all replicas' steps
        assert sec == 3.0 and steps == 30.0
    # the pooled estimate obeys the counting theorem
    lc, S, rv = replicas.estimates(res[0][1], 2)
    ex = np.array(exact_counts[2][:13], dtype=float)
    for n in range(4):
        assert math.isclose(math.exp(lc[n]), ex[n], rel_tol=1e-12)
    z = (np.exp(lc - np.log(ex)) - 1.0)[4:] / np.sqrt(rv[4:])
    assert np.max(np.abs(z)) < 4.5, z


@pytest.mark.parametrize("d,n_max", [(2, 14), (3, 10)])
def test_estimates_from_one_run_match_the_oracle(d, n_max):
    """Without a process group the pooled estimate is the single run's: the same
    numbers as the oracle's own estimates from its tables."""
    h = orc.Oracle(d, n_max, 3, seed=7)
    h.run(200)
    t = h.tables()
    lc, S, rv = replicas.estimates(replicas.pool_tables(dict(W=t["W"], S=t["S"], Q=t["Q"], M=t["M"])), d)
    lo, So, rvo = h.estimates()
    assert np.array_equal(S, So)
    assert np.allclose(lc, lo, rtol=1e-13, atol=1e-12)
    assert np.allclose(rv, rvo, rtol=1e-10, atol=0)


def test_without_a_group_the_timing_is_local():
    assert replicas.reduce_timing(2.5, 7) == (2.5, 7.0)
