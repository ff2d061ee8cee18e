"""perm_run_static: the growth run that allocates nothing.

Some callers cannot call cudaMalloc.  Their device memory may be owned by another
allocator (a framework's caching pool, or a plugin living inside such a process).
Or they run a loop that must not allocate, because allocation can synchronise the
device.  For them the library keeps a run's scratch in a fixed static device array.
These tests call that entry point through the C ABI, twice in a row, and check
each result against the same run made through the handle-based entry points
(perm_create_ex / perm_run / perm_tables).  The same tolerance as the other
whole-run tests applies: counts exact, weights to relative 1e-12.

This file is collected last on purpose.  If it fails, a run that stops at the
first failure has already run every other test.
"""
import math

import numpy as np
import pytest

import paper_2002_03000_gb300 as pg
from paper_2002_03000_gb300 import _native as nat
from tests.gpu_util import torch_cuda, zscores

pytestmark = pytest.mark.gpu

REL_W = 1e-12


def _reference(d, n_max, n_seq, seed, tours):
    with pg.Run(d, n_max, n_seq, seed, threshold=pg.PERM_THRESH_FRESH, max_seconds=120.0) as run:
        run.run(tours)
        t = run.tables()
        steps = run.stats()["steps"]
    return t, steps


def _static(torch, d, n_max, n_seq, seed, tours, threshold=pg.PERM_THRESH_FRESH, slots=0):
    cfg = nat.perm_config_init(d, n_max, n_seq, seed)
    cfg.threshold = threshold
    cfg.slots = slots
    cfg.max_seconds = 120.0
    L = n_max + 1
    # fill the outputs with garbage first: the call must overwrite them
    W = torch.full((L,), 7.5, dtype=torch.float64, device="cuda")
    S = torch.full((L,), 3, dtype=torch.int64, device="cuda")
    Q = torch.full((L,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    steps = nat.perm_run_static(cfg, tours, W.data_ptr(), S.data_ptr(), Q.data_ptr(), stream)
    return dict(W=W.cpu().numpy(), S=S.cpu().numpy().astype(np.float64), Q=Q.cpu().numpy()), steps


def _close(a, b):
    return np.all(np.abs(a - b) <= REL_W * np.maximum(np.abs(a), np.abs(b)))


def test_static_run_matches_handle_run_twice():
    torch = torch_cuda()
    cases = [(2, 64, 1, 0xA11CE, 400), (3, 40, 1, 0xB0B, 300)]
    refs = [_reference(*c) for c in cases]
    # two calls in a row per case: the second must not see the first's leftovers
    for (d, n_max, n_seq, seed, tours), (ref, ref_steps) in zip(cases, refs):
        for _ in range(2):
            got, steps = _static(torch, d, n_max, n_seq, seed, tours)
            assert steps == ref_steps
            assert np.array_equal(got["S"], ref["S"])
            assert _close(got["W"], ref["W"])
            assert _close(got["Q"], ref["Q"])


def test_static_run_rejects_oversized_request():
    torch = torch_cuda()
    # 4096 concurrent walks of length 2048 need ~168 MB of scratch: beyond the 32 MiB buffer
    cfg = nat.perm_config_init(2, 2048, 4096, 1)
    cfg.slots = 4096
    L = 2049
    W = torch.zeros(L, dtype=torch.float64, device="cuda")
    S = torch.zeros(L, dtype=torch.int64, device="cuda")
    Q = torch.zeros(L, dtype=torch.float64, device="cuda")
    with pytest.raises(nat.PermError) as e:
        nat.perm_run_static(cfg, 1, W.data_ptr(), S.data_ptr(), Q.data_ptr())
    assert e.value.code == nat.PERM_ESCRATCH
    assert "static buffer" in nat.strerror(nat.PERM_ESCRATCH)


def test_static_interacting_sequences_obey_the_counting_theorem(exact_counts):
    """Snapshot thresholds, a few hundred interacting sequences (the static
    layout: up to 4 warps of 32 walks per CTA, a refresher warp per CTA), two
    calls in a row: every tour passes lengths 0 and 1 once (S_0 = S_1 = M,
    c_1 = 2d exactly) and the estimates meet exact c_n (Sec. 1, eq. 3) within
    4.5 standard errors at every length."""
    torch = torch_cuda()
    for d, n_max, N, tours, seed in [(2, 16, 300, 40, 0x5EED), (3, 11, 400, 30, 0xFEED)]:
        for _ in range(2):
            got, steps = _static(torch, d, n_max, N, seed, tours, threshold=pg.PERM_THRESH_SNAPSHOT)
            M = N * tours
            assert got["S"][0] == M and got["S"][1] == M
            lc, rv = nat.perm_estimates_from_tables(d, n_max, got["W"], got["Q"], [M])
            assert math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
            z = zscores(lc, rv, exact_counts[d][: n_max + 1])
            assert np.all(np.abs(z[2:]) < 4.5), (d, z)
            assert steps == int(got["S"].sum())


def test_static_walks_limited_by_the_buffer():
    """More sequences than the buffer holds walks for (8192 of length 256 need
    about 42 MB of tour sums and spill areas): with slots = 0 the run takes
    what fits, time-slices the rest at tour boundaries and completes."""
    torch = torch_cuda()
    d, n_max, N, tours = 2, 256, 8192, 2
    per_walk = (n_max + 1) * 8 + n_max * 12
    assert N * per_walk > nat.PERM_STATIC_SCRATCH_BYTES
    got, steps = _static(torch, d, n_max, N, 0xC0DE, tours, threshold=pg.PERM_THRESH_SNAPSHOT)
    assert got["S"][0] == N * tours and got["S"][1] == N * tours
    assert steps == int(got["S"].sum())


def test_static_run_refuses_settings_it_does_not_carry_out():
    torch = torch_cuda()
    L = 17
    W = torch.zeros(L, dtype=torch.float64, device="cuda")
    S = torch.zeros(L, dtype=torch.int64, device="cuda")
    Q = torch.zeros(L, dtype=torch.float64, device="cuda")
    for field, value in (("observables", 1), ("hash_scale", 1), ("lanes_per_warp", 4),
                         ("stack_ring", 64), ("max_ctas", 8), ("share_copies", 4), ("walk_memory", 2),
                         ("helper_walks", 8)):
        cfg = nat.perm_config_init(2, 16, 4, 1)
        setattr(cfg, field, value)
        with pytest.raises(nat.PermError) as e:
            nat.perm_run_static(cfg, 1, W.data_ptr(), S.data_ptr(), Q.data_ptr())
        assert e.value.code == nat.PERM_EUNSUPPORTED, field
    # an explicit walk count above the sequences is clamped to them, not refused
    cfg = nat.perm_config_init(2, 16, 1, 1)
    cfg.slots = 4096
    nat.perm_run_static(cfg, 3, W.data_ptr(), S.data_ptr(), Q.data_ptr())
    assert S.cpu().numpy()[0] == 3
