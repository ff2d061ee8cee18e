"""Batched flatPERM runs: many independent runs grown by one CUDA-graph launch
(per-run kernels on streams, or one persistent kernel for all runs).

Thin wrapper of perm_batch_* (include/perm.h); the runs' growth happens in the
persistent CUDA kernel, the graph is captured and replayed by the library.
"""
from __future__ import annotations

import math

import numpy as np

from . import _native as nat


class Batch:
    """R independent runs; run() replays the captured graph (fresh tables).

    persistent=False: one growth kernel per run on up to 64 streams;
    persistent=True: one persistent kernel on every SM grows all runs (CTAs move
    between runs as their tours run out)."""

    def __init__(self, configs, tours, n_streams=0, persistent=False):
        self.run_cfgs = list(configs)
        self.tours = [int(t) for t in tours]
        self.persistent = bool(persistent)
        if self.persistent:
            self.b = nat.perm_batch_create_persistent(self.run_cfgs, self.tours)
        else:
            self.b = nat.perm_batch_create(self.run_cfgs, self.tours, n_streams)

    def run(self):
        nat.perm_batch_run(self.b)

    def continue_runs(self, extra_tours):
        """More tours per sequence for each run on top of its tables (0: leave it)."""
        nat.perm_batch_continue(self.b, extra_tours)

    def run_to_target(self, target, first_tours=None, max_rounds=8, max_tours=1 << 16):
        """Every run until the relative standard error of its c_{n_max} is at most
        `target`: a replay from empty tables (the creation-time tours), then
        continuations that give each run still above its target the tours the
        1/tours law of the variance predicts it needs (at least 4 more, at most
        8 times what it has), until all meet it or `max_rounds`.  Returns the
        tours per sequence each run grew and the rounds taken."""
        self.run()
        tours = list(self.tours)
        for rnd in range(max_rounds):
            extra = [more_tours(self.estimates(r)[2][cfg.n_max], tours[r], target, max_tours)
                     for r, cfg in enumerate(self.run_cfgs)]
            if not any(extra):
                return tours, rnd
            self.continue_runs(extra)
            tours = [t + e for t, e in zip(tours, extra)]
        return tours, max_rounds

    def estimates(self, r):
        return nat.perm_batch_estimates(self.b, r, self.run_cfgs[r].n_max)

    def stats(self, r):
        return nat.perm_batch_stats(self.b, r)

    def close(self):
        if self.b:
            nat.perm_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def more_tours(relvar, tours, target, max_tours=1 << 16):
    """Tours per sequence to add to a run with `tours` whose c_{n_max} has relative
    variance `relvar`, to bring its relative standard error to `target`: 0 when
    met; else what the 1/tours law of the variance predicts (10% over), at least
    4 and at most 8 times what it has."""
    rel = math.sqrt(relvar) if relvar >= 0 and math.isfinite(relvar) else float("inf")
    if rel <= target or tours >= max_tours:
        return 0
    want = tours * ((rel / target) ** 2 - 1.0) if math.isfinite(rel) else tours
    return int(min(max(math.ceil(1.1 * want), 4), 8 * tours, max_tours - tours))


def make_config(d, n_max, n_seq, seed, run_id=0, **kw):
    cfg = nat.perm_config_init(d, n_max, n_seq, seed)
    cfg.run_id = run_id
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def mixed_runs(count=96, seed=1, n_max_range=(64, 2048), n_seq_range=(256, 8192)):
    """Seeded workload of independent runs: d uniform in {2, 3}, n_max and the
    number of sequences log-uniform in the given ranges (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r in range(count):
        d = int(rng.integers(2, 4))
        n_max = int(round(math.exp(rng.uniform(math.log(n_max_range[0]), math.log(n_max_range[1])))))
        n_seq = int(round(math.exp(rng.uniform(math.log(n_seq_range[0]), math.log(n_seq_range[1])))))
        out.append((d, n_max, n_seq))
    return out


def autotune(cfg, probe_tours=2):
    """Pick walks per warp, hash size and stack ring for cfg by short calibration
    runs at equal work (written into cfg)."""
    return nat.perm_autotune(cfg, probe_tours)
