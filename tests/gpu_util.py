"""Helpers for the GPU tests: device buffers via torch, calls through the C ABI."""
import numpy as np

from oracle import oracle as orc
from paper_2002_03000_gb300 import _native as nat

REL_W = 1e-12    # weights: relative tolerance against the oracle

# Relative-error floor for nearly deterministic lengths.  With many concurrent
# walks and shared snapshot thresholds, the per-tour variance misses the
# correlation that a common threshold induces between tours; it matters only
# where the intrinsic variance is tiny (n = 2: estimated 2.9e-6 against a
# spread of 7.6e-6 over 20 seeds of 4096 x 8 tours; at n >= 3 the two agree).
SIGMA_FLOOR = 1e-5




def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


# |x - r| <= 6.01 2^-24 x for the kernel's single-precision estimate x of r
# (the bound derived beside ratio_estimate); the tests allow 2^-21.
REL_R_ESTIMATE = 2.0 ** -21


def debug_step(states, d, n_max, seed, run_id=0, force_exact=0):
    """Run the growth step of the CUDA path on snapshot states (list of dicts
    from tests.inputs) through perm_debug_step; returns host numpy arrays
    (out_i with 11 columns: outcome, a_plus, free_mask, c, dirs[6], exact; r;
    child weight)."""
    torch = torch_cuda()
    B = len(states)
    L = n_max + 1
    coords = np.zeros((B, L, d), dtype=np.int32)
    length = np.zeros(B, dtype=np.int32)
    for b, st in enumerate(states):
        w = st["walk"]
        coords[b, : w.shape[0]] = w
        length[b] = w.shape[0] - 1
    dev = "cuda"
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt, device=dev)
    c_t = t(coords.reshape(-1), torch.int32)
    l_t = t(length, torch.int32)
    W_t = t(np.array([s["W"] for s in states], dtype=np.float64), torch.float64)
    S_t = t(np.array([s["Wsum"] for s in states], dtype=np.float64), torch.float64)
    u64 = lambda key: np.array([s[key] for s in states], dtype=np.uint64).view(np.int64)
    u32 = lambda key: np.array([s[key] for s in states], dtype=np.uint32).view(np.int32)
    M_t = t(u64("M"), torch.int64)
    o_t = t(u64("ordinal"), torch.int64)
    s_t = t(u32("seq"), torch.int32)
    u_t = t(u32("tour"), torch.int32)
    out_i = torch.zeros(B * 11, dtype=torch.int32, device=dev)
    out_r = torch.zeros(B, dtype=torch.float64, device=dev)
    out_w = torch.zeros(B, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    nat.perm_debug_step(d, n_max, B, c_t.data_ptr(), l_t.data_ptr(), W_t.data_ptr(), S_t.data_ptr(),
                        M_t.data_ptr(), o_t.data_ptr(), s_t.data_ptr(), u_t.data_ptr(), seed, run_id,
                        force_exact, out_i.data_ptr(), out_r.data_ptr(), out_w.data_ptr(), stream)
    torch.cuda.synchronize()
    return out_i.cpu().numpy().reshape(B, 11), out_r.cpu().numpy(), out_w.cpu().numpy()


def same_step(got, ref):
    """The kernel's node against the oracle's: outcome, a_+, free mask, c and the
    chosen steps exactly; r bit for bit where the kernel evaluated it exactly,
    else within the estimate's bound; the children's weight to REL_W."""
    ok = (got["outcome"] == ref["outcome"] and got["a_plus"] == ref["a_plus"] and
          got["free_mask"] == ref["free_mask"] and got["c"] == ref["c"] and
          list(got["dirs"]) == list(ref["dirs"]))
    if ref["outcome"] >= 2:
        if got["exact"]:
            ok &= got["r"] == ref["r"]
        else:
            ok &= abs(got["r"] - ref["r"]) <= REL_R_ESTIMATE * ref["r"]
    if ref["outcome"] == 3:
        ok &= abs(got["child_w"] - ref["child_w"]) <= REL_W * abs(ref["child_w"])
    return bool(ok)


def debug_philox(ctrs, key):
    torch = torch_cuda()
    ctr = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1)
    B = ctr.size // 4
    c_t = torch.as_tensor(ctr.view(np.int32)).cuda()
    out = torch.zeros(B * 4, dtype=torch.int32, device="cuda")
    nat.perm_debug_philox(B, c_t.data_ptr(), key, out.data_ptr())
    return out.cpu().numpy().view(np.uint32).reshape(B, 4)


def Run(*args, **kw):
    """pg.Run with a short per-launch time bound for tests."""
    import paper_2002_03000_gb300 as pg
    kw.setdefault("max_seconds", 120.0)
    return pg.Run(*args, **kw)


def zscores(lc, rv, exact):
    """z-scores of the estimates against exact c_n; an estimate that is exact
    with zero estimated variance (short lengths, where every weight is equal)
    scores 0."""
    ex = np.array(exact, dtype=float)
    rel = np.exp(lc[: len(ex)] - np.log(ex)) - 1.0
    rv = rv[: len(ex)]
    exact_zero = (np.abs(rel) < 1e-12) & (rv == 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        z = rel / np.sqrt(rv + SIGMA_FLOOR ** 2)
    return np.where(exact_zero, 0.0, z)


def replay(recs, coords, d, n_max, seed):
    """Replay sampled nodes of a real run in the oracle, each from the state the
    node saw (walk, W, Wsum, M); returns the mismatches."""
    bad = []
    for rec, co in zip(recs, coords):
        n = rec.n
        ref = orc.step(d, n_max, co[: n + 1], rec.W, rec.Wsum, int(rec.M), int(rec.ordinal),
                       int(rec.seq), int(rec.tour), seed)
        got = dict(outcome=rec.outcome, a_plus=rec.a_plus, free_mask=rec.free_mask, c=rec.c,
                   dirs=list(rec.dirs[: max(rec.c, 0)]), exact=rec.exact, r=rec.r,
                   child_w=rec.child_w)
        if not same_step(got, ref):
            bad.append((n, rec.outcome, ref))
    return bad
