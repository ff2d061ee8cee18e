"""Served flatPERM: continuous batching of estimation requests on one GPU.

A request asks for the estimates of c_n up to n_max on the square or cubic
lattice until the relative standard error of c_{n_max} is at most `target`.
The server:
  - admits requests in arrival order while the device-memory budget and the
    number of resident runs allow (a run's stacks and tables stay resident
    until it retires);
  - grows every resident run in chunks of tours on its own CUDA stream, so
    chunks of different requests overlap on the device;
  - polls chunk completion without blocking, reads the estimates of finished
    chunks, retires runs that meet their target (freeing their memory and
    slot) and queues the next chunk of the others.
Latency = retirement time - arrival time.  The growth itself runs in the CUDA
kernels behind the C ABI; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import deque

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    d: int
    n_max: int
    target: float                 # relative standard error of c_{n_max}
    arrival: float                # seconds from the start of the session
    n_seq: int = 1024
    seed: int = 1
    threshold: int = 0            # PERM_THRESH_SNAPSHOT (0) or PERM_THRESH_FRESH (1)
    chunk_tours: int = 8
    max_tours: int = 1 << 20      # give up (retire unmet) after this many tours per sequence
    # filled in by the server
    admitted: float = float("nan")
    retired: float = float("nan")
    tours: int = 0
    steps: int = 0
    rel_se: float = float("inf")
    log_cn: np.ndarray = None
    relvar: np.ndarray = None     # relative variance of every c_n, when the engine gives it
    met: bool = False


class Server:
    """Continuous-batching scheduler over an engine (the GPU engine below, or a
    fake one in CPU tests)."""

    def __init__(self, engine, hbm_budget_bytes=120e9, max_resident=16, clock=time.perf_counter):
        self.engine = engine
        self.budget = float(hbm_budget_bytes)
        self.max_resident = int(max_resident)
        self.clock = clock
        self.waiting = deque()
        self.resident = {}            # rid -> (request, job)
        self.done = []
        self.bytes_in_use = 0.0
        self.t0 = None
        self.peak_bytes = 0.0
        self.peak_resident = 0

    def now(self):
        return self.clock() - self.t0

    def _admit(self):
        while self.waiting and len(self.resident) < self.max_resident:
            req = self.waiting[0]
            need = self.engine.bytes_needed(req)
            if self.bytes_in_use + need > self.budget:
                break
            self.waiting.popleft()
            job = self.engine.start(req)
            req.admitted = self.now()
            self.bytes_in_use += job.bytes
            self.peak_bytes = max(self.peak_bytes, self.bytes_in_use)
            self.resident[req.rid] = (req, job)
            self.peak_resident = max(self.peak_resident, len(self.resident))
            self.engine.queue_chunk(job, req.chunk_tours)

    def _poll(self):
        for rid in list(self.resident):
            req, job = self.resident[rid]
            if not self.engine.chunk_done(job):
                continue
            req.tours += req.chunk_tours
            log_cn, rel_se, steps = self.engine.read(job)
            req.log_cn, req.rel_se, req.steps = log_cn, rel_se, steps
            req.relvar = getattr(job, "relvar", None)
            if rel_se <= req.target or req.tours >= req.max_tours:
                req.met = rel_se <= req.target
                req.retired = self.now()
                self.engine.stop(job)
                self.bytes_in_use -= job.bytes
                del self.resident[rid]
                self.done.append(req)
            else:
                self.engine.queue_chunk(job, req.chunk_tours)

    def serve(self, requests, deadline_s=None, idle_sleep=2e-4):
        """Serve requests (arrival times in seconds from now); returns them."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self.t0 = self.clock()
        i = 0
        while i < len(pending) or self.waiting or self.resident:
            t = self.now()
            while i < len(pending) and pending[i].arrival <= t:
                self.waiting.append(pending[i])
                i += 1
            self._poll()
            self._admit()
            if deadline_s is not None and t > deadline_s:
                break
            if idle_sleep:
                time.sleep(idle_sleep)
        return self.done

    @staticmethod
    def summary(done, wall_s):
        lat = np.array([r.retired - r.arrival for r in done]) if done else np.zeros(0)
        steps = sum(r.steps for r in done)
        return {
            "requests": len(done),
            "met": int(sum(r.met for r in done)),
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "steps": int(steps),
            "steps_per_s": steps / wall_s if wall_s > 0 else None,
        }


class _Job:
    def __init__(self, run, stream, event, nbytes):
        self.run, self.stream, self.event, self.bytes = run, stream, event, nbytes


class GpuEngine:
    """Runs requests as library handles, each on its own CUDA stream."""

    def __init__(self, max_ctas=-1, lanes_per_warp=0):
        import torch
        from . import Run, _native
        self.torch, self.Run, self.nat = torch, Run, _native
        self.max_ctas = max_ctas
        self.lanes_per_warp = lanes_per_warp
        self.bytes_est = {}

    def bytes_needed(self, req):
        # tables + per-walk tour sums (two rows per walk) and stack spill areas (an upper estimate)
        L = req.n_max + 1
        return 3 * 8 * L + req.n_seq * (16 * L + 12 * req.n_max) + (1 << 20)

    def start(self, req):
        torch = self.torch
        run = self.Run(req.d, req.n_max, req.n_seq, req.seed, run_id=req.rid,
                       threshold=req.threshold, max_ctas=self.max_ctas,
                       lanes_per_warp=self.lanes_per_warp, max_seconds=600.0)
        stream = torch.cuda.Stream()
        run.set_stream(stream.cuda_stream)
        nbytes = run.stats()["device_bytes"]
        return _Job(run, stream, torch.cuda.Event(), nbytes)

    def queue_chunk(self, job, tours):
        self.nat.perm_run(job.run.h, tours)
        job.event.record(job.stream)

    def chunk_done(self, job):
        return job.event.query()

    def read(self, job):
        lc, S, rv = job.run.estimates()
        job.relvar = rv
        n_max = job.run.n_max
        st = job.run.stats()
        if st["status"] != 0:
            raise RuntimeError("request run failed: %s" % self.nat.strerror(st["status"]))
        return lc, math.sqrt(rv[n_max]), st["steps"]

    def stop(self, job):
        job.run.close()


def poisson_requests(count, rate_per_s, seed=1, n_max_range=(64, 1024), targets=(1e-3, 1e-4),
                     n_seq=1024):
    """Seeded request stream: Poisson arrivals, d uniform in {2, 3}, n_max
    log-uniform, target drawn uniformly from `targets`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        d = int(rng.integers(2, 4))
        n_max = int(round(math.exp(rng.uniform(math.log(n_max_range[0]), math.log(n_max_range[1])))))
        target = float(targets[int(rng.integers(0, len(targets)))])
        out.append(Request(rid=rid, d=d, n_max=n_max, target=target, arrival=t, n_seq=n_seq,
                           seed=seed))
    return out
