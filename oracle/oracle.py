"""ctypes wrapper around the C oracle (test infrastructure only).

Every function returns numpy arrays; nothing here does any of the method's
arithmetic -- it only marshals arguments to ``perm_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import numpy as np

from . import build as _build

ORC_ALG1 = 1
ORC_ALG2 = 2
OUTCOMES = {0: "leaf_nmax", 1: "trapped", 2: "pruned", 3: "children"}

_lib = None


def configure(L):
    """Declare the C signatures on a loaded oracle library."""
    u32p = C.POINTER(C.c_uint32)
    L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.orc_philox4x32_10.restype = None
    L.orc_enumerate.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int64)]
    L.orc_enumerate_r2.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.orc_scale_exp.argtypes = [C.c_int, C.c_int]
    L.orc_ratio.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int64]
    L.orc_ratio.restype = C.c_double
    L.orc_step.argtypes = [
        C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int32), C.c_double, C.c_double,
        C.c_int64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32,
        C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double),
        C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.orc_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int,
                             C.c_uint64, C.c_uint32, C.c_int]
    L.orc_run.argtypes = [C.c_void_p, C.c_int64]
    L.orc_run_threads.argtypes = [C.c_void_p, C.c_int64, C.c_int]
    L.orc_set_cutoffs.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.c_int, C.c_double]
    dp = C.POINTER(C.c_double)
    i64p = C.POINTER(C.c_int64)
    L.orc_tables.argtypes = [C.c_void_p, dp, dp, dp, i64p, i64p, i64p]
    L.orc_estimates.argtypes = [C.c_void_p, dp, dp, dp]
    L.orc_observable_r2.argtypes = [C.c_void_p, dp]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_destroy.restype = None
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = configure(C.CDLL(_build.build()))
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def enumerate_cn(d: int, n: int) -> np.ndarray:
    out = np.zeros(n + 1, dtype=np.int64)
    rc = lib().orc_enumerate(d, n, _p(out, C.c_int64))
    if rc != 0:
        raise ValueError("orc_enumerate failed: %d" % rc)
    return out


def enumerate_r2(d: int, n: int):
    """(c_k, sum over walks of length k of |omega_k|^2) for k = 0..n, exact."""
    c = np.zeros(n + 1, dtype=np.int64)
    r2 = np.zeros(n + 1, dtype=np.int64)
    rc = lib().orc_enumerate_r2(d, n, _p(c, C.c_int64), _p(r2, C.c_int64))
    if rc != 0:
        raise ValueError("orc_enumerate_r2 failed: %d" % rc)
    return c, r2


def scale_exp(d: int, n: int) -> int:
    return lib().orc_scale_exp(d, n)


def ratio(n: int, W: float, Wsum: float, M: int) -> float:
    """r = W / [W_n]^sample with [W_n]^sample = (Wsum + W) / M (Sec. 2, eq. 6)."""
    return float(lib().orc_ratio(n, W, Wsum, M))


def step(d, n_max, coords, W, Wsum, M, ordinal, seq, tour, seed, run=0):
    """Growth step of one node on a snapshot walk (coords: (n+1, d) int).  W is
    the node's weight, Wsum the sum of the weights recorded at its length before
    it, M the tours started."""
    co = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1)
    n = co.size // d - 1
    a = C.c_int(0); mask = C.c_int(0); r = C.c_double(0); c = C.c_int(0)
    dirs = (C.c_int * 6)()
    cw = C.c_double(0)
    rc = lib().orc_step(d, n_max, n, _p(co, C.c_int32), W, Wsum, M, ordinal, seq, tour,
                        seed, run, C.byref(a), C.byref(mask), C.byref(r), C.byref(c),
                        dirs, C.byref(cw))
    if rc < 0:
        raise ValueError("orc_step rejected the state: %d" % rc)
    return dict(outcome=rc, a_plus=a.value, free_mask=mask.value, r=r.value,
                c=c.value, dirs=[dirs[i] for i in range(c.value)], child_w=cw.value)


class Oracle:
    """A flatPERM simulation on the CPU (Alg. 2 shared table, or Alg. 1)."""

    def __init__(self, d, n_max, n_seq, seed, run=0, alg=ORC_ALG2):
        self.d, self.n_max, self.n_seq, self.alg = d, n_max, n_seq, alg
        h = C.c_void_p()
        rc = lib().orc_create(C.byref(h), d, n_max, n_seq, seed, run, alg)
        if rc != 0:
            raise ValueError("orc_create failed: %d" % rc)
        self._h = h

    def set_cutoffs(self, T_hi, t_lo, copies=2, q=2.0):
        """Original PERM (Sec. 2): cut-offs per length at the stored scale (None,
        None: back to flatPERM)."""
        if T_hi is None and t_lo is None:
            rc = lib().orc_set_cutoffs(self._h, None, None, 0, 0.0)
        else:
            hi = np.ascontiguousarray(T_hi, dtype=np.float64)
            lo = np.ascontiguousarray(t_lo, dtype=np.float64)
            assert hi.shape == lo.shape == (self.n_max + 1,)
            rc = lib().orc_set_cutoffs(self._h, _p(hi, C.c_double), _p(lo, C.c_double), int(copies), float(q))
        if rc != 0:
            raise RuntimeError("orc_set_cutoffs failed: %d" % rc)

    def run(self, tours_per_seq):
        rc = lib().orc_run(self._h, tours_per_seq)
        if rc != 0:
            raise RuntimeError("orc_run failed: %d" % rc)

    def run_threads(self, tours_per_seq, threads):
        """Algorithm 2 on `threads` host threads sharing the table (Sec. 3)."""
        rc = lib().orc_run_threads(self._h, tours_per_seq, threads)
        if rc != 0:
            raise RuntimeError("orc_run_threads failed: %d" % rc)

    def tables(self):
        ntab = self.n_seq if self.alg == ORC_ALG1 else 1
        L = (self.n_max + 1) * ntab
        W = np.zeros(L); S = np.zeros(L); Q = np.zeros(L)
        M = np.zeros(ntab, dtype=np.int64)
        steps = C.c_int64(0); ms = C.c_int64(0)
        lib().orc_tables(self._h, _p(W, C.c_double), _p(S, C.c_double), _p(Q, C.c_double),
                         _p(M, C.c_int64), C.byref(steps), C.byref(ms))
        return dict(W=W, S=S, Q=Q, M=M, steps=steps.value, max_stack=ms.value)

    def r2_table(self):
        """Raw sum of W |omega_n|^2 per length (rows as in tables())."""
        ntab = self.n_seq if self.alg == ORC_ALG1 else 1
        R = np.zeros((self.n_max + 1) * ntab)
        lib().orc_observable_r2(self._h, _p(R, C.c_double))
        return R

    def mean_r2(self):
        """<|omega_n|^2> by the ratio estimator (Sec. 1, eq. 5): R_n / W_n (Alg. 1:
        the average over sequences of R/M divided by that of W/M)."""
        t = self.tables()
        R = self.r2_table()
        L = self.n_max + 1
        ntab = self.n_seq if self.alg == ORC_ALG1 else 1
        M = t["M"].astype(float)
        num = sum(R[i * L:(i + 1) * L] / M[i] for i in range(ntab))
        den = sum(t["W"][i * L:(i + 1) * L] / M[i] for i in range(ntab))
        with np.errstate(divide="ignore", invalid="ignore"):
            return num / den

    def estimates(self):
        L = self.n_max + 1
        lc = np.zeros(L); S = np.zeros(L); rv = np.zeros(L)
        lib().orc_estimates(self._h, _p(lc, C.c_double), _p(S, C.c_double), _p(rv, C.c_double))
        return lc, S, rv

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
