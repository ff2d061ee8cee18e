"""Host logic of the continuous-batching server, with a fake engine (no GPU):
admission respects the memory budget and the resident cap, requests that arrive
while others run are admitted as slots free up, runs retire at their target,
and latencies are arrival-to-retirement."""
import numpy as np

from paper_2002_03000_gb300.serve import Request, Server


class FakeJob:
    def __init__(self, req, nbytes):
        self.req, self.bytes = req, nbytes
        self.chunks_queued = 0
        self.chunks_read = 0


class FakeEngine:
    """Each chunk 'finishes' on the next poll; the relative error after k
    chunks is e0 / sqrt(k) with e0 set per request."""

    def __init__(self, nbytes=10.0):
        self.nbytes = nbytes
        self.live = 0
        self.max_live = 0

    def bytes_needed(self, req):
        return self.nbytes

    def start(self, req):
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return FakeJob(req, self.nbytes)

    def queue_chunk(self, job, tours):
        job.chunks_queued += 1

    def chunk_done(self, job):
        return job.chunks_queued > job.chunks_read

    def read(self, job):
        job.chunks_read += 1
        e0 = 0.1 * (1 + job.req.rid % 3)
        return np.zeros(job.req.n_max + 1), e0 / np.sqrt(job.chunks_read), 100 * job.chunks_read

    def stop(self, job):
        self.live -= 1


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


def _requests(n, spacing=0.0005, target=0.02):
    return [Request(rid=i, d=2 + i % 2, n_max=64, target=target, arrival=i * spacing) for i in range(n)]


def test_admission_respects_budget_and_cap():
    eng = FakeEngine(nbytes=10.0)
    srv = Server(eng, hbm_budget_bytes=35.0, max_resident=5, clock=FakeClock())
    done = srv.serve(_requests(20), idle_sleep=0)
    assert len(done) == 20 and all(r.met for r in done)
    assert eng.max_live <= 3                  # 35 bytes / 10 per run
    assert srv.peak_bytes <= 35.0
    srv2 = Server(FakeEngine(nbytes=1.0), hbm_budget_bytes=1e9, max_resident=4, clock=FakeClock())
    srv2.serve(_requests(20), idle_sleep=0)
    assert srv2.peak_resident == 4


def test_continuous_admission_and_retirement_targets():
    eng = FakeEngine()
    srv = Server(eng, hbm_budget_bytes=1e9, max_resident=3, clock=FakeClock())
    reqs = _requests(12, spacing=0.0002)
    done = srv.serve(reqs, idle_sleep=0)
    # e0 in {0.1, 0.2, 0.3} and target 0.02 -> (e0 / 0.02)^2 chunks: 25, 100, 225
    for r in done:
        e0 = 0.1 * (1 + r.rid % 3)
        assert r.met and r.rel_se <= r.target
        k = 1
        while e0 / np.sqrt(k) > r.target:     # chunks the fake engine needs
            k += 1
        assert r.tours == k * r.chunk_tours
        assert r.retired >= r.admitted >= r.arrival
    # later arrivals were admitted while earlier ones were still running
    admits = sorted(r.admitted for r in done)
    retires = sorted(r.retired for r in done)
    assert admits[3] < retires[-1]
    s = Server.summary(done, wall_s=1.0)
    assert s["requests"] == 12 and s["met"] == 12 and s["p99_latency_s"] >= s["p50_latency_s"]


def test_unmet_requests_retire_at_the_tour_cap():
    eng = FakeEngine()
    srv = Server(eng, clock=FakeClock())
    req = Request(rid=0, d=2, n_max=64, target=1e-9, arrival=0.0, max_tours=40)
    done = srv.serve([req], idle_sleep=0)
    assert len(done) == 1 and not done[0].met and done[0].tours == 40


def test_batch_target_rule():
    """The tour rule of the to-target drivers: nothing once the target is met,
    else the 1/tours law of the variance (10% over), at least 4 and at most 8
    times what the run has; and the Batch wrapper keeps its methods."""
    from paper_2002_03000_gb300 import batch as pb
    assert pb.more_tours(0.01 ** 2, 16, 0.02) == 0
    assert pb.more_tours(0.04 ** 2, 16, 0.03) == 14          # ceil(1.1 x 16 x (16/9 - 1))
    assert pb.more_tours(0.1 ** 2, 16, 0.01) == 128          # capped at 8 times the tours
    assert pb.more_tours(0.0301 ** 2, 100, 0.03) == 4        # at least 4
    assert pb.more_tours(float("inf"), 8, 0.01) == 9           # unknown variance: 1.1 x the tours
    for name in ("run", "continue_runs", "run_to_target", "estimates", "stats", "close", "__enter__"):
        assert hasattr(pb.Batch, name), name
