"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/perm.h (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_2002_03000_gb300 import _native, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "perm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(perm_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_t")))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(_native.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the Python binding binds all of them, under the same names
    assert sorted(_native.EXPORTS) == names


def test_strerror_and_config_defaults(lib):
    L = _native.load()
    assert L.perm_strerror(0) == b"ok"
    assert b"invalid" in L.perm_strerror(-1)
    cfg = _native.perm_config_init(2, 512, 4096, 1)
    assert (cfg.d, cfg.n_max, cfg.n_seq, cfg.seed, cfg.alg, cfg.threshold) == (2, 512, 4096, 1, 2, 0)


def test_argument_checks_need_no_device(lib):
    L = _native.load()
    h = ctypes.c_void_p()
    # invalid arguments are rejected before any device call
    assert L.perm_create(ctypes.byref(h), 4, 10, 1, 1) == _native.PERM_EINVAL
    assert L.perm_create(ctypes.byref(h), 2, 0, 1, 1) == _native.PERM_EINVAL
    assert L.perm_create(ctypes.byref(h), 2, 10, 0, 1) == _native.PERM_EINVAL
    assert L.perm_run(None, 5) == _native.PERM_EINVAL
    assert L.perm_debug_step(2, 600, 1, *([None] * 8), 0, 0, 0, *([None] * 3), None) == _native.PERM_EINVAL
    L.perm_destroy(None)   # NULL-safe


def test_cutoff_and_batch_argument_checks_need_no_device(lib):
    L = _native.load()
    b = ctypes.c_void_p()
    # original PERM cut-offs: a NULL handle is rejected
    assert L.perm_set_cutoffs(None, None, None, 2, 2.0) == _native.PERM_EINVAL
    # batches: no runs, or a negative tour count, are rejected before any device call
    cfg = (_native.perm_config * 1)(_native.perm_config_init(2, 16, 4, 1))
    tours = (ctypes.c_int64 * 1)(-1)
    assert L.perm_batch_create(ctypes.byref(b), cfg, tours, 0, 0) == _native.PERM_EINVAL
    assert L.perm_batch_create(ctypes.byref(b), cfg, tours, 1, 0) == _native.PERM_EINVAL
    assert L.perm_batch_create_persistent(ctypes.byref(b), cfg, tours, 0) == _native.PERM_EINVAL
    assert L.perm_batch_create_persistent(ctypes.byref(b), cfg, tours, 1) == _native.PERM_EINVAL
    # the persistent form takes Algorithm-2 snapshot runs only
    alg1 = _native.perm_config_init(2, 16, 4, 1)
    alg1.alg = _native.PERM_ALG1
    cfg1 = (_native.perm_config * 1)(alg1)
    ok_tours = (ctypes.c_int64 * 1)(2)
    assert L.perm_batch_create_persistent(ctypes.byref(b), cfg1, ok_tours, 1) == _native.PERM_EUNSUPPORTED
    L.perm_batch_destroy(None)   # NULL-safe


def test_checkpoint_files_are_checked_before_any_device_call(lib, tmp_path):
    L = _native.load()
    h = ctypes.c_void_p()
    assert L.perm_save(None, b"x") == _native.PERM_EINVAL
    assert L.perm_load(ctypes.byref(h), str(tmp_path / "missing.ckpt").encode()) == _native.PERM_EINVAL
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint" * 64)
    assert L.perm_load(ctypes.byref(h), str(bad).encode()) == _native.PERM_EINVAL
    assert not h.value
    assert L.perm_get_config(None, None) == _native.PERM_EINVAL
