"""ctypes binding of libperm.so: the C ABI of include/perm.h, same names.

Argument marshalling only -- every step of the growth path runs in the CUDA
kernels of csrc/.  Loading fails loudly when the library is missing or the
device cannot run it; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libperm.so")

PERM_OK = 0
PERM_EINVAL = -1
PERM_ENOMEM = -2
PERM_EOVERFLOW = -3
PERM_EDEVICE = -4
PERM_ETIMEOUT = -5
PERM_EUNSUPPORTED = -6
PERM_ESCRATCH = -7
PERM_STATIC_SCRATCH_BYTES = 32 << 20
PERM_ALG1 = 1
PERM_ALG2 = 2
PERM_THRESH_SNAPSHOT = 0
PERM_THRESH_FRESH = 1

# every exported symbol declared in include/perm.h
EXPORTS = (
    "perm_config_init", "perm_create", "perm_create_ex", "perm_set_stream", "perm_run", "perm_reset",
    "perm_run_sync", "perm_estimates", "perm_tables", "perm_stats", "perm_trace_enable",
    "perm_trace_read", "perm_destroy", "perm_strerror", "perm_debug_step", "perm_debug_philox",
    "perm_run_static", "perm_set_cutoffs", "perm_save", "perm_load", "perm_get_config", "perm_batch_create", "perm_batch_create_persistent", "perm_batch_run", "perm_batch_size",
    "perm_batch_estimates", "perm_batch_stats", "perm_batch_destroy", "perm_autotune",
    "perm_observable_r2", "perm_estimates_from_tables", "perm_batch_continue",
)
PERM_COMBINE_MEAN = 0
PERM_COMBINE_GEOMETRIC = 1


class perm_config(C.Structure):
    _fields_ = [("d", C.c_int), ("n_max", C.c_int), ("n_seq", C.c_int), ("seed", C.c_uint64),
                ("run_id", C.c_uint32), ("alg", C.c_int), ("threshold", C.c_int),
                ("slots", C.c_int), ("lanes_per_warp", C.c_int), ("refresh_ns", C.c_int),
                ("max_seconds", C.c_double), ("ramp_c0", C.c_int), ("ramp_gamma", C.c_double),
                ("max_ctas", C.c_int), ("hash_scale", C.c_int), ("share_copies", C.c_int),
                ("stack_ring", C.c_int), ("observables", C.c_int), ("walk_memory", C.c_int),
                ("helper_walks", C.c_int)]


class perm_stats_t(C.Structure):
    _fields_ = [("steps", C.c_int64), ("tours", C.c_int64), ("max_stack", C.c_int64),
                ("copies", C.c_int64), ("refreshes", C.c_int64), ("iterations", C.c_int64),
                ("slots", C.c_int), ("ctas", C.c_int), ("lanes_per_warp", C.c_int),
                ("warps_per_cta", C.c_int), ("hash_slots", C.c_int), ("status", C.c_int),
                ("device_bytes", C.c_int64), ("tours_finished", C.c_int64),
                ("shared", C.c_int64), ("exact_steps", C.c_int64), ("walk_memory", C.c_int),
                ("pad", C.c_int)]


class perm_trace_record(C.Structure):
    _fields_ = [("n", C.c_int32), ("a_plus", C.c_int32), ("free_mask", C.c_int32),
                ("c", C.c_int32), ("outcome", C.c_int32), ("exact", C.c_int32),
                ("dirs", C.c_int32 * 6), ("seq", C.c_uint32), ("tour", C.c_uint32),
                ("ordinal", C.c_uint64), ("M", C.c_uint64), ("W", C.c_double),
                ("Wsum", C.c_double), ("r", C.c_double), ("child_w", C.c_double)]


class PermError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libperm.so and declare the signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libperm.so not built: run paper_2002_03000_gb300.build.build() "
                          "(expected at %s)" % path)
    L = C.CDLL(path)
    vp, i64, u64, u32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32
    hp = C.POINTER(C.c_void_p)
    dp = C.POINTER(C.c_double)
    L.perm_config_init.argtypes = [C.POINTER(perm_config), C.c_int, C.c_int, C.c_int, u64]
    L.perm_config_init.restype = None
    L.perm_create.argtypes = [hp, C.c_int, C.c_int, C.c_int, u64]
    L.perm_create_ex.argtypes = [hp, C.POINTER(perm_config)]
    L.perm_set_stream.argtypes = [vp, vp]
    L.perm_run.argtypes = [vp, i64]
    L.perm_run_sync.argtypes = [vp, i64]
    L.perm_reset.argtypes = [vp]
    L.perm_estimates.argtypes = [vp, dp, dp, dp]
    L.perm_estimates_from_tables.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, C.POINTER(i64),
                                             C.c_int, dp, dp]
    L.perm_observable_r2.argtypes = [vp, dp, dp]
    L.perm_tables.argtypes = [vp, dp, dp, dp, C.POINTER(i64)]
    L.perm_stats.argtypes = [vp, C.POINTER(perm_stats_t)]
    L.perm_trace_enable.argtypes = [vp, i64, i64, C.c_int]
    L.perm_trace_read.argtypes = [vp, C.POINTER(i64), C.POINTER(perm_trace_record),
                                  C.POINTER(C.c_int32)]
    L.perm_destroy.argtypes = [vp]
    L.perm_destroy.restype = None
    L.perm_strerror.argtypes = [C.c_int]
    L.perm_strerror.restype = C.c_char_p
    L.perm_debug_step.argtypes = [C.c_int, C.c_int, C.c_int] + [vp] * 8 + [u64, u32, C.c_int] + [vp] * 3 + [vp]
    L.perm_debug_philox.argtypes = [C.c_int, vp, C.POINTER(u32), vp]
    L.perm_run_static.argtypes = [C.POINTER(perm_config), i64, vp, vp, vp, C.POINTER(i64), vp]
    L.perm_batch_create.argtypes = [hp, C.POINTER(perm_config), C.POINTER(i64), C.c_int, C.c_int]
    L.perm_set_cutoffs.argtypes = [vp, dp, dp, C.c_int, C.c_double]
    L.perm_save.argtypes = [vp, C.c_char_p]
    L.perm_load.argtypes = [hp, C.c_char_p]
    L.perm_get_config.argtypes = [vp, C.POINTER(perm_config)]
    L.perm_batch_create_persistent.argtypes = [hp, C.POINTER(perm_config), C.POINTER(i64), C.c_int]
    L.perm_batch_run.argtypes = [vp]
    L.perm_batch_continue.argtypes = [vp, C.POINTER(i64)]
    L.perm_batch_size.argtypes = [vp]
    L.perm_batch_estimates.argtypes = [vp, C.c_int, dp, dp, dp]
    L.perm_batch_stats.argtypes = [vp, C.c_int, C.POINTER(perm_stats_t)]
    L.perm_batch_destroy.argtypes = [vp]
    L.perm_batch_destroy.restype = None
    L.perm_autotune.argtypes = [C.POINTER(perm_config), i64]
    for name in EXPORTS:
        if name not in ("perm_config_init", "perm_destroy", "perm_strerror", "perm_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return load().perm_strerror(code).decode()
    except Exception:
        return "error %d" % code


def _check(code, what):
    if code != PERM_OK:
        raise PermError(code, what)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def perm_config_init(d, n_max, n_seq, seed):
    cfg = perm_config()
    load().perm_config_init(C.byref(cfg), d, n_max, n_seq, seed)
    return cfg


def perm_create(d, n_max, n_seq, seed):
    h = C.c_void_p()
    _check(load().perm_create(C.byref(h), d, n_max, n_seq, seed), "perm_create")
    return h


def perm_create_ex(cfg: perm_config):
    h = C.c_void_p()
    _check(load().perm_create_ex(C.byref(h), C.byref(cfg)), "perm_create_ex")
    return h


def perm_set_stream(h, stream_ptr: int):
    _check(load().perm_set_stream(h, C.c_void_p(stream_ptr)), "perm_set_stream")


def perm_run(h, tours_per_seq: int):
    _check(load().perm_run(h, tours_per_seq), "perm_run")


def perm_run_sync(h, tours_per_seq: int):
    _check(load().perm_run_sync(h, tours_per_seq), "perm_run_sync")


def perm_reset(h):
    _check(load().perm_reset(h), "perm_reset")


def perm_estimates_from_tables(d, n_max, W, Q, M, combine=PERM_COMBINE_MEAN):
    """(log c_n, relative variance) from raw tables at the stored scale: W, Q of
    shape (rows, n_max+1) or (n_max+1,), Q may be None; M one count per row."""
    W = np.ascontiguousarray(W, dtype=np.float64).reshape(-1)
    rows = W.size // (n_max + 1)
    if rows < 1 or rows * (n_max + 1) != W.size:
        raise ValueError("W must hold whole rows of n_max+1")
    Qa = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64).reshape(-1)
    if Qa is not None and Qa.size != W.size:
        raise ValueError("Q must match W")
    Ma = np.ascontiguousarray(M, dtype=np.int64).reshape(-1)
    if Ma.size != rows:
        raise ValueError("one tour count per row")
    lc = np.zeros(n_max + 1)
    rv = np.zeros(n_max + 1)
    _check(load().perm_estimates_from_tables(d, n_max, rows, _dp(W), None if Qa is None else _dp(Qa),
                                             Ma.ctypes.data_as(C.POINTER(C.c_int64)), combine,
                                             _dp(lc), _dp(rv)), "perm_estimates_from_tables")
    return lc, rv


def perm_estimates(h, n_max: int):
    L = n_max + 1
    lc, S, rv = np.empty(L), np.empty(L), np.empty(L)
    _check(load().perm_estimates(h, _dp(lc), _dp(S), _dp(rv)), "perm_estimates")
    return lc, S, rv


def perm_observable_r2(h, n_max: int, rows: int = 1):
    """(mean |omega_n|^2 by eq. 5, raw sums of W |omega_n|^2 per length and row)."""
    L = n_max + 1
    mean = np.empty(L)
    raw = np.empty(L * rows)
    _check(load().perm_observable_r2(h, _dp(mean), _dp(raw)), "perm_observable_r2")
    return mean, raw


def perm_tables(h, n_max: int, rows: int = 1):
    L = (n_max + 1) * rows
    W, S, Q = np.empty(L), np.empty(L), np.empty(L)
    M = np.zeros(rows, dtype=np.int64)
    _check(load().perm_tables(h, _dp(W), _dp(S), _dp(Q), M.ctypes.data_as(C.POINTER(C.c_int64))),
           "perm_tables")
    return dict(W=W, S=S, Q=Q, M=M)


def perm_stats(h) -> dict:
    st = perm_stats_t()
    _check(load().perm_stats(h, C.byref(st)), "perm_stats")
    return {name: getattr(st, name) for name, _ in perm_stats_t._fields_}


def perm_trace_enable(h, every: int, tour_every: int, capacity: int):
    _check(load().perm_trace_enable(h, every, tour_every, capacity), "perm_trace_enable")


def perm_trace_read(h, capacity: int, n_max: int, d: int):
    count = C.c_int64(0)
    recs = (perm_trace_record * max(capacity, 1))()
    coords = np.zeros(max(capacity, 1) * (n_max + 1) * d, dtype=np.int32)
    _check(load().perm_trace_read(h, C.byref(count), recs,
                                  coords.ctypes.data_as(C.POINTER(C.c_int32))), "perm_trace_read")
    kept = min(count.value, capacity)
    return count.value, [recs[i] for i in range(kept)], coords.reshape(-1, n_max + 1, d)[:kept]


def perm_destroy(h):
    if h:
        load().perm_destroy(h)


def perm_debug_step(d, n_max, B, coords, length, W, Wsum, M, ordinal, seq, tour, seed, run_id,
                    force_exact, out_i, out_r, out_w, stream=0):
    """All array arguments are device pointers (ints), e.g. tensor.data_ptr()."""
    _check(load().perm_debug_step(d, n_max, B, coords, length, W, Wsum, M, ordinal, seq, tour,
                                  seed, run_id, force_exact, out_i, out_r, out_w, stream),
           "perm_debug_step")


def perm_run_static(cfg, tours_per_seq, W_dev, S_dev, Q_dev, stream=0):
    """One growth run with the library's static scratch (no allocation).  W_dev,
    S_dev, Q_dev are device pointers of n_max+1 float64/uint64/float64 entries.
    Returns the number of growth steps."""
    steps = C.c_int64(0)
    _check(load().perm_run_static(C.byref(cfg), tours_per_seq, W_dev, S_dev, Q_dev,
                                  C.byref(steps), stream), "perm_run_static")
    return steps.value


def perm_batch_create(cfgs, tours, n_streams=0):
    """cfgs: list of perm_config; tours: list of tours per sequence."""
    R = len(cfgs)
    arr = (perm_config * R)(*cfgs)
    t = (C.c_int64 * R)(*[int(x) for x in tours])
    b = C.c_void_p()
    _check(load().perm_batch_create(C.byref(b), arr, t, R, n_streams), "perm_batch_create")
    return b


def perm_save(h, path):
    """Checkpoint the run at its current tour boundary."""
    _check(load().perm_save(h, os.fsencode(path)), "perm_save")


def perm_load(path):
    """A new handle continuing a checkpointed run."""
    h = C.c_void_p()
    _check(load().perm_load(C.byref(h), os.fsencode(path)), "perm_load")
    return h


def perm_get_config(h):
    cfg = perm_config()
    _check(load().perm_get_config(h, C.byref(cfg)), "perm_get_config")
    return cfg


def perm_set_cutoffs(h, T_hi, t_lo, copies=2, q=2.0):
    """Original PERM cut-offs (stored scale, n_max+1 each); None, None: flatPERM."""
    if T_hi is None and t_lo is None:
        _check(load().perm_set_cutoffs(h, None, None, 0, 0.0), "perm_set_cutoffs")
        return
    hi = np.ascontiguousarray(T_hi, dtype=np.float64)
    lo = np.ascontiguousarray(t_lo, dtype=np.float64)
    if hi.shape != lo.shape:
        raise ValueError("cut-off arrays differ in length")
    _check(load().perm_set_cutoffs(h, _dp(hi), _dp(lo), int(copies), float(q)), "perm_set_cutoffs")


def perm_batch_create_persistent(cfgs, tours):
    """The same batch grown by one persistent launch (Alg. 2, snapshot runs only)."""
    R = len(cfgs)
    arr = (perm_config * R)(*cfgs)
    t = (C.c_int64 * R)(*[int(x) for x in tours])
    b = C.c_void_p()
    _check(load().perm_batch_create_persistent(C.byref(b), arr, t, R), "perm_batch_create_persistent")
    return b


def perm_batch_run(b):
    _check(load().perm_batch_run(b), "perm_batch_run")


def perm_batch_continue(b, extra_tours):
    arr = (C.c_int64 * len(extra_tours))(*[int(t) for t in extra_tours])
    _check(load().perm_batch_continue(b, arr), "perm_batch_continue")


def perm_batch_estimates(b, r, n_max):
    L = n_max + 1
    lc, S, rv = np.empty(L), np.empty(L), np.empty(L)
    _check(load().perm_batch_estimates(b, r, _dp(lc), _dp(S), _dp(rv)), "perm_batch_estimates")
    return lc, S, rv


def perm_batch_stats(b, r):
    st = perm_stats_t()
    _check(load().perm_batch_stats(b, r, C.byref(st)), "perm_batch_stats")
    return {name: getattr(st, name) for name, _ in perm_stats_t._fields_}


def perm_batch_destroy(b):
    if b:
        load().perm_batch_destroy(b)


def perm_autotune(cfg, probe_tours):
    _check(load().perm_autotune(C.byref(cfg), probe_tours), "perm_autotune")
    return cfg


def perm_debug_philox(B, ctr_dev, key, out_dev):
    k = (C.c_uint32 * 2)(int(key[0]), int(key[1]))
    _check(load().perm_debug_philox(B, ctr_dev, k, out_dev), "perm_debug_philox")
