"""One persistent launch growing many runs (CTAs move between runs).

The scheduling of a persistent batch differs from a run made alone, so its
tables are compared by what holds for any schedule: every tour is counted at
lengths 0 and 1, c_1 = 2d exactly, the counting theorem (Sec. 2: the weight sum
over M tours estimates c_n without bias) against exact counts, and agreement
in law with the same run made alone."""
import math

import numpy as np
import pytest

import paper_2002_03000_gb300 as pg
from paper_2002_03000_gb300 import batch as pb
from paper_2002_03000_gb300 import _native as nat
from tests.gpu_util import SIGMA_FLOOR, torch_cuda

pytestmark = pytest.mark.gpu


def _check_run(lc, S, rv, d, n, M, exact_counts, k=5.0):
    assert S[0] == M and S[1] == M
    assert math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)
    ex = np.array(exact_counts[d][: min(n, 11 if d == 3 else 16) + 1], dtype=float)
    rel = np.exp(lc[: len(ex)] - np.log(ex)) - 1
    sig = np.sqrt(rv[: len(ex)] + 1e-10)
    assert np.all(np.abs(rel[2:]) < k * sig[2:]), (rel, sig)


SPEC = [(2, 16, 300, 40), (3, 11, 500, 20), (2, 256, 1000, 8), (3, 600, 700, 4), (2, 1024, 256, 4),
        (3, 64, 3000, 6), (2, 48, 64, 50)]


def test_persistent_batch_counting_theorem_and_replay(exact_counts):
    torch_cuda()
    cfgs = [pb.make_config(d, n, N, 7 + i, max_seconds=120.0) for i, (d, n, N, _) in enumerate(SPEC)]
    with pb.Batch(cfgs, [t for *_, t in SPEC], persistent=True) as b:
        for replay in range(2):          # each replay starts every run from empty tables
            b.run()
            for r, (d, n, N, t) in enumerate(SPEC):
                st = b.stats(r)
                assert st["status"] == 0
                assert st["tours_finished"] == N * t
                lc, S, rv = b.estimates(r)
                _check_run(lc, S, rv, d, n, N * t, exact_counts)


def test_persistent_batch_agrees_with_alone():
    """The same run in a persistent batch and alone (other seeds): log c_n agree
    within the combined standard errors.  The z-scores of neighbouring lengths are
    strongly correlated (one tour's fluctuation moves all of them), so their mean
    over lengths is about one standard normal draw: both it and the largest |z|
    get bounds that a real bias of a few standard errors breaks."""
    torch_cuda()
    spec = [(2, 200, 2000, 8), (3, 150, 1500, 8), (2, 64, 500, 30)]
    cfgs = [pb.make_config(d, n, N, 31 + i, max_seconds=120.0) for i, (d, n, N, _) in enumerate(spec)]
    with pb.Batch(cfgs, [t for *_, t in spec], persistent=True) as b:
        b.run()
        for r, (d, n, N, t) in enumerate(spec):
            lcb, Sb, rvb = b.estimates(r)
            with pg.Run(d, n, N, 131 + r, max_seconds=120.0) as run:
                run.run(t)
                lca, Sa, rva = run.estimates()
            ok = np.isfinite(lca) & np.isfinite(lcb) & (rva > 0) & (rvb > 0)
            z = (lcb[ok] - lca[ok]) / np.sqrt(rva[ok] + rvb[ok] + 2 * SIGMA_FLOOR ** 2)
            assert np.max(np.abs(z)) < 5.0, (r, np.max(np.abs(z)))
            assert abs(np.mean(z)) < 3.5, (r, np.mean(z))


def test_persistent_batch_mixed_workload_completes():
    """A seeded mix of square and cubic runs of very different sizes: every run
    finishes all its tours (runs outnumber what one CTA each could start at once)."""
    torch_cuda()
    runs = pb.mixed_runs(40, seed=3, n_max_range=(32, 700), n_seq_range=(64, 2048))
    cfgs = [pb.make_config(d, n, N, 1, run_id=i, max_seconds=120.0) for i, (d, n, N) in enumerate(runs)]
    with pb.Batch(cfgs, [3] * len(runs), persistent=True) as b:
        b.run()
        for r, (d, n, N) in enumerate(runs):
            st = b.stats(r)
            assert st["status"] == 0, (r, runs[r], st)
            assert st["tours_finished"] == 3 * N
            lc, S, rv = b.estimates(r)
            assert S[0] == 3 * N and math.isclose(math.exp(lc[1]), 2 * d, rel_tol=1e-12)


def test_persistent_batch_without_shared_copies(exact_counts):
    torch_cuda()
    spec = [(2, 16, 300, 40), (3, 11, 500, 20), (2, 128, 800, 6)]
    cfgs = [pb.make_config(d, n, N, 17 + i, max_seconds=120.0, share_copies=-1)
            for i, (d, n, N, _) in enumerate(spec)]
    with pb.Batch(cfgs, [t for *_, t in spec], persistent=True) as b:
        b.run()
        for r, (d, n, N, t) in enumerate(spec):
            assert b.stats(r)["status"] == 0 and b.stats(r)["shared"] == 0
            lc, S, rv = b.estimates(r)
            _check_run(lc, S, rv, d, n, N * t, exact_counts)


def test_persistent_batch_rejects_other_forms():
    torch_cuda()
    fresh = pb.make_config(2, 32, 1, 1, threshold=pg.PERM_THRESH_FRESH)
    alg1 = pb.make_config(2, 32, 16, 1, alg=pg.PERM_ALG1)
    for c in (fresh, alg1):
        with pytest.raises(nat.PermError) as ei:
            pb.Batch([c], [2], persistent=True)
        assert ei.value.code == nat.PERM_EUNSUPPORTED
