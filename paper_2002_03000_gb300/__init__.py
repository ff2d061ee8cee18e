"""GB300-native interacting flatPERM (Campbell and Janse van Rensburg, "Parallel PERM").

The growth step runs in the CUDA kernels of ``csrc/`` behind the C ABI of
``include/perm.h`` (libperm.so).  ``_native`` binds that ABI with the same
names; ``Run`` is a small convenience wrapper around one handle.
"""
from . import _native
from ._native import (PERM_ALG1, PERM_ALG2, PERM_THRESH_FRESH, PERM_THRESH_SNAPSHOT,  # noqa: F401
                      PermError, perm_config_init)


class Run:
    """One flatPERM run (a perm_handle): create, run tours, read estimates."""

    def __init__(self, d, n_max, n_seq, seed, run_id=0, alg=PERM_ALG2,
                 threshold=PERM_THRESH_SNAPSHOT, slots=0, lanes_per_warp=0, refresh_ns=0,
                 max_seconds=0.0, ramp_c0=0, ramp_gamma=0.0, max_ctas=0, hash_scale=0,
                 share_copies=0, stack_ring=0, observables=0, walk_memory=0, helper_walks=0):
        cfg = _native.perm_config_init(d, n_max, n_seq, seed)
        cfg.run_id = run_id
        cfg.alg = alg
        cfg.threshold = threshold
        cfg.slots = slots
        cfg.lanes_per_warp = lanes_per_warp
        cfg.refresh_ns = refresh_ns
        cfg.max_seconds = max_seconds
        cfg.ramp_c0 = ramp_c0
        cfg.ramp_gamma = ramp_gamma
        cfg.max_ctas = max_ctas
        cfg.hash_scale = hash_scale
        cfg.share_copies = share_copies
        cfg.stack_ring = stack_ring
        cfg.observables = observables
        cfg.walk_memory = walk_memory
        cfg.helper_walks = helper_walks
        self.d, self.n_max, self.n_seq, self.alg = d, n_max, n_seq, alg
        self.h = _native.perm_create_ex(cfg)

    def save(self, path):
        """Checkpoint at the current tour boundary (see perm_save)."""
        _native.perm_save(self.h, path)

    @classmethod
    def load(cls, path):
        """A Run continuing the checkpoint at `path` (see perm_load)."""
        self = cls.__new__(cls)
        self.h = None
        self.h = _native.perm_load(path)
        cfg = _native.perm_get_config(self.h)
        self.d, self.n_max, self.n_seq, self.alg = cfg.d, cfg.n_max, cfg.n_seq, cfg.alg
        return self

    def set_cutoffs(self, T_hi, t_lo, copies=2, q=2.0):
        """Original PERM (Sec. 2) from now on: enrich into `copies` copies above
        T_hi[n], prune with probability 1 - 1/q below t_lo[n] (both n_max+1
        values at the stored weight scale); None, None: back to flatPERM."""
        if T_hi is not None or t_lo is not None:
            if len(T_hi) != self.n_max + 1 or len(t_lo) != self.n_max + 1:
                raise ValueError("cut-offs need n_max + 1 values each")
        _native.perm_set_cutoffs(self.h, T_hi, t_lo, copies, q)

    def run(self, tours_per_seq, sync=True):
        if sync:
            _native.perm_run_sync(self.h, tours_per_seq)
        else:
            _native.perm_run(self.h, tours_per_seq)

    def reset(self):
        _native.perm_reset(self.h)

    def set_stream(self, stream_ptr):
        _native.perm_set_stream(self.h, stream_ptr)

    def estimates(self):
        return _native.perm_estimates(self.h, self.n_max)

    def mean_r2(self):
        """<|omega_n|^2> by the ratio estimator (Sec. 1, eq. 5) and the raw sums
        (needs observables=1 at creation)."""
        rows = self.n_seq if self.alg == PERM_ALG1 else 1
        return _native.perm_observable_r2(self.h, self.n_max, rows)

    def tables(self):
        rows = self.n_seq if self.alg == PERM_ALG1 else 1
        return _native.perm_tables(self.h, self.n_max, rows)

    def stats(self):
        return _native.perm_stats(self.h)

    def trace_enable(self, every, tour_every=1, capacity=1024):
        self._trace_cap = capacity
        _native.perm_trace_enable(self.h, every, tour_every, capacity)

    def trace_read(self):
        return _native.perm_trace_read(self.h, self._trace_cap, self.n_max, self.d)

    def close(self):
        if self.h:
            _native.perm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
