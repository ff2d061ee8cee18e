"""Batched (one CUDA-graph launch for many runs) and served (continuous
batching) forms against the same runs made alone.

Runs with fresh thresholds and one sequence are deterministic, so a run's
tables are the same alone, in a batch and in a served mix: counts exactly,
weights to relative 1e-12.  Interacting runs (snapshot thresholds, many
sequences) are checked by their exact invariants and the counting theorem."""
import math

import numpy as np
import pytest

import paper_2002_03000_gb300 as pg
from paper_2002_03000_gb300 import batch as pb
from paper_2002_03000_gb300 import serve as ps
from tests.gpu_util import Run, torch_cuda, zscores

pytestmark = pytest.mark.gpu

REL_W = 1e-12


def _close(a, b):
    return np.all(np.abs(a - b) <= REL_W * np.maximum(np.abs(a), np.abs(b)))


def _alone(d, n_max, seed, tours):
    with Run(d, n_max, 1, seed, threshold=pg.PERM_THRESH_FRESH) as run:
        run.run(tours)
        return run.estimates(), run.tables()


FRESH_RUNS = [(2, 40, 11, 300), (3, 30, 12, 200), (2, 100, 13, 60), (3, 700, 14, 8), (2, 16, 15, 900)]


def test_batch_equals_alone_and_replays():
    torch_cuda()
    cfgs = [pb.make_config(d, n, 1, s, threshold=pg.PERM_THRESH_FRESH, max_seconds=120.0)
            for d, n, s, _ in FRESH_RUNS]
    tours = [t for *_, t in FRESH_RUNS]
    alone = [_alone(d, n, s, t) for d, n, s, t in FRESH_RUNS]
    with pb.Batch(cfgs, tours) as b:
        for replay in range(2):          # a replay starts every run again from empty tables
            b.run()
            for r, (d, n, s, t) in enumerate(FRESH_RUNS):
                lc, S, rv = b.estimates(r)
                (lc0, S0, rv0), t0 = alone[r]
                assert np.array_equal(S, S0)
                fin = np.isfinite(lc0)
                assert np.allclose(lc[fin], lc0[fin], rtol=0, atol=1e-12)
                assert b.stats(r)["status"] == 0


def test_batch_of_interacting_runs(exact_counts):
    torch_cuda()
    spec = [(2, 16, 300, 40), (3, 11, 500, 20), (2, 256, 1000, 8), (3, 600, 700, 4), (2, 1024, 256, 4)]
    cfgs = [pb.make_config(d, n, N, 7 + i, max_seconds=120.0) for i, (d, n, N, _) in enumerate(spec)]
    with pb.Batch(cfgs, [t for *_, t in spec]) as b:
        b.run()
        for r, (d, n, N, t) in enumerate(spec):
            lc, S, rv = b.estimates(r)
            M = N * t
            assert S[0] == M and S[1] == M
            assert math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
            # shared thresholds correlate the tours, so the per-tour variance
            # understates the spread at the shortest lengths: a relative floor on
            # sigma there, and 5 sigma over all runs and lengths
            z = zscores(lc, rv, exact_counts[d][: min(n, 11 if d == 3 else 16) + 1])
            assert np.all(np.abs(z[2:]) < 5.0), (r, z)


def test_autotune_picks_a_runnable_layout():
    torch_cuda()
    cfg = pb.make_config(2, 128, 512, 3, max_seconds=60.0)
    pb.autotune(cfg, probe_tours=2)
    assert cfg.lanes_per_warp in (0, 2, 4, 8, 16, 32) and cfg.hash_scale in (0, 1)
    assert cfg.stack_ring in (16, 64)
    run = pg.Run(2, 128, 512, 3, lanes_per_warp=cfg.lanes_per_warp, hash_scale=cfg.hash_scale,
                 stack_ring=cfg.stack_ring, max_seconds=60.0)
    run.run(4)
    assert run.stats()["status"] == 0
    run.close()


def test_served_results_equal_alone():
    torch_cuda()
    # a burst of deterministic requests (one sequence, fresh thresholds): each
    # retires after a number of chunks fixed by its own estimates, so its final
    # tables are the same served in the mix as grown alone
    reqs = []
    for i in range(10):
        d = 2 + i % 2
        reqs.append(ps.Request(rid=i, d=d, n_max=24 + 4 * i, target=0.05, arrival=0.002 * i,
                               n_seq=1, seed=100 + i, threshold=pg.PERM_THRESH_FRESH, chunk_tours=40,
                               max_tours=4000))
    srv = ps.Server(ps.GpuEngine(max_ctas=8), hbm_budget_bytes=4e9, max_resident=4)
    done = srv.serve(reqs)
    assert len(done) == 10 and all(r.met for r in done)
    assert srv.peak_resident >= 2                    # runs overlapped on the device
    for r in done:
        with Run(r.d, r.n_max, 1, r.seed, run_id=r.rid, threshold=pg.PERM_THRESH_FRESH) as run:
            run.run(r.tours)
            lc, S, rv = run.estimates()
        fin = np.isfinite(lc)
        assert np.allclose(r.log_cn[fin], lc[fin], rtol=0, atol=1e-12)
        assert math.isclose(math.sqrt(rv[r.n_max]), r.rel_se, rel_tol=1e-9)


def test_served_interacting_requests_meet_exact_counts_and_the_oracle(exact_counts):
    """A burst of interacting requests served together as the benchmark serves
    them (snapshot thresholds, 512-1024 sequences each, continuous batching on
    densely packed CTAs), at lengths where c_n is known exactly (n_max 16 on the
    square lattice, 11 on the cubic).  Every retired request meets its target,
    its estimates agree with exact c_n (Sec. 1, eq. 3) within 4.5 standard errors
    at every length, and with an independent run of the CPU oracle within 4.5
    combined standard errors."""
    from oracle import oracle as orc
    torch_cuda()
    reqs = []
    for i in range(12):
        d = 2 + i % 2
        reqs.append(ps.Request(rid=i, d=d, n_max=16 if d == 2 else 11, target=5e-3,
                               arrival=0.003 * i, n_seq=512 if i % 3 else 1024, seed=200 + i,
                               chunk_tours=4, max_tours=2000))
    srv = ps.Server(ps.GpuEngine(max_ctas=-1), hbm_budget_bytes=120e9, max_resident=8)
    done = srv.serve(reqs)
    assert len(done) == 12 and all(r.met for r in done)
    assert srv.peak_resident >= 2
    ref = {}
    for d, n_max in ((2, 16), (3, 11)):
        o = orc.Oracle(d, n_max, 12, seed=4242)
        o.run(3000)
        lc, S, rv = o.estimates()
        ref[d] = (lc, rv)
    for r in done:
        lc, rv = r.log_cn, r.relvar
        z = zscores(lc, rv, exact_counts[r.d][: r.n_max + 1])
        assert np.all(np.abs(z[2:]) < 4.5), (r.rid, z)
        lco, rvo = ref[r.d]
        zo = (lc - lco)[2:] / np.sqrt(rv[2:] + rvo[2:] + 1e-10)
        assert np.all(np.abs(zo) < 4.5), (r.rid, zo)


def test_batch_continue_equals_runs_alone():
    """A streams batch of deterministic runs (one sequence, fresh thresholds)
    replayed and then continued run by run equals each run grown alone by the
    same total tours; a run given no extra tours keeps its tables; a later replay
    starts every run again from its creation-time tours."""
    torch_cuda()
    spec = [(2, 40, 21, 100, 60), (3, 30, 22, 80, 0), (2, 64, 23, 50, 25)]
    cfgs = [pb.make_config(d, n, 1, s, threshold=pg.PERM_THRESH_FRESH, max_seconds=120.0)
            for d, n, s, _, _ in spec]
    with pb.Batch(cfgs, [t for *_, t, _ in spec]) as b:
        b.run()
        before = [b.estimates(r) for r in range(len(spec))]
        b.continue_runs([e for *_, e in spec])
        for r, (d, n, s, t, e) in enumerate(spec):
            (lc0, S0, rv0), _ = _alone(d, n, s, t + e)
            lc, S, rv = b.estimates(r)
            assert np.array_equal(S, S0), r
            fin = np.isfinite(lc0)
            assert np.allclose(lc[fin], lc0[fin], rtol=0, atol=1e-12), r
            if e == 0:
                assert np.array_equal(S, before[r][1])
        b.run()
        for r, (d, n, s, t, e) in enumerate(spec):
            assert np.array_equal(b.estimates(r)[1], before[r][1]), r


def test_persistent_batch_runs_to_target(exact_counts):
    """A persistent batch driven to a common target error: every run meets it,
    tours grown on top of the first replay add up (S_0 = M exactly), and the
    estimates stay within 5 standard errors of exact c_n."""
    torch_cuda()
    spec = [(2, 16, 300), (3, 11, 400), (2, 16, 600), (3, 11, 200)]
    cfgs = [pb.make_config(d, n, N, 31 + i, max_seconds=120.0) for i, (d, n, N) in enumerate(spec)]
    with pb.Batch(cfgs, [8] * len(spec), persistent=True) as b:
        tours, rounds = b.run_to_target(3e-3)
        assert 1 <= rounds < 8
        for r, (d, n, N) in enumerate(spec):
            lc, S, rv = b.estimates(r)
            assert math.sqrt(rv[n]) <= 3e-3, r
            assert S[0] == N * tours[r] and S[1] == N * tours[r]
            z = zscores(lc, rv, exact_counts[d][: n + 1])
            assert np.all(np.abs(z[2:]) < 5.0), (r, z)
