#!/usr/bin/env python3
"""Benchmark: walk-growth steps/s of interacting flatPERM (Algorithm 2) on GB300.

Workload (one "step" = one complete run from empty tables): square lattice,
n_max = 512, 4096 interacting sequences x 256 tours each, shared FP64 tables,
Philox4x32-10 seed 1 -- synthetic by construction (the lattice is the input).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun each rank runs an independent replica
(distinct run id) on its own GPU; value = all ranks' steps / max time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walk-growth steps/s and time to 1e-4 rel. error in c_n (1 GB300) vs plain form"
UNIT = "steps/s"
WORKLOAD = dict(d=2, n_max=512, n_seq=4096, tours=256, seed=1)
WORKLOAD_NAME = "plain massively parallel flatPERM, d=2, n_max=512, 4096 sequences x 256 tours"
L2_FLUSH_BYTES = 512 << 20
# c_0..c_16 of the square lattice (exact; self-avoiding walk counts)
EXACT_C_SQUARE = [1, 4, 12, 36, 100, 284, 780, 2172, 5916, 16268, 44100, 120292, 324932,
                  881500, 2374444, 6416596, 17245332]


def bytes_per_step(d, f):
    """Algorithmic bytes one growth step moves: 2d probes of k-byte keys, insert and
    LIFO delete, the site's coordinates, the W_n/S_n update and W_n read, the per-tour
    sum read+write, and a 16-byte stack push+pop per extra copy (f per step)."""
    k = 4
    base = 2 * d * k + 2 * k + 4 * d + 16 + 8 + 16
    return base + 32.0 * f


KERNEL_SOURCES = ("perm_kernels.cu", "perm_kernels.cuh", "perm_device.cuh")


def code_tokens(text):
    """The code of a C++/CUDA source without its comments and with whitespace
    runs collapsed, so that a changed comment does not count as a changed
    kernel (the sources hold no string literal with a comment marker)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sources_sha256(texts=None):
    """SHA-256 over the code (comments dropped) of the growth kernel's sources;
    texts: the sources' contents in KERNEL_SOURCES order (default: the files)."""
    import hashlib
    h = hashlib.sha256()
    if texts is None:
        texts = []
        for name in KERNEL_SOURCES:
            with open(os.path.join(ROOT, "paper_2002_03000_gb300", "csrc", name), encoding="utf-8") as f:
                texts.append(f.read())
    for t in texts:
        h.update(code_tokens(t).encode("utf-8"))
        h.update(b"\0")
    return h.hexdigest()


def measured_counters():
    """From the ncu capture summarised in profiles/ (if taken on the current kernel
    sources): DRAM bytes (read + write) of one growth-kernel launch of this workload
    and warp instructions per growth step; (None, None, why) otherwise (a stale count
    would mislead)."""
    import re
    path = os.path.join(ROOT, "profiles", "grow_kernel_c2_traffic.md")
    try:
        text = open(path).read()
    except OSError:
        return None, None, "no capture"
    b = re.search(r"^bytes_per_launch:\s*(\d+)\s*$", text, re.M)
    i = re.search(r"^warp_inst_per_step:\s*([0-9.]+)\s*$", text, re.M)
    h = re.search(r"^kernel_sources_sha256:\s*([0-9a-f]{64})\s*$", text, re.M)
    if not b or not h:
        return None, None, "capture summary unreadable"
    if h.group(1) != kernel_sources_sha256():
        return None, None, "kernel changed since the capture"
    return (int(b.group(1)), float(i.group(1)) if i else None,
            "ncu capture of the current kernel (profiles/grow_kernel_c2_traffic.md)")


def sm_count():
    try:
        import torch
        return torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        return 152


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        import tempfile
        out_dir = os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, "bench_clocks_%d.csv" % index)

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(seconds=15.0):
    """The oracle, as it stands, on the host cores: Algorithm 2 on every host core
    (the paper's own form, Sec. 3: threads growing sequences that share the table,
    updated atomically), the benchmark workload from empty tables in rounds of 8
    tours per sequence until `seconds` of work; and the sequential oracle (one
    thread) for a third of that."""
    from oracle import oracle as orc
    w = WORKLOAD
    cores = host_cores()
    o = orc.Oracle(w["d"], w["n_max"], w["n_seq"], w["seed"])
    t0 = time.perf_counter()
    rounds = 0
    while True:
        o.run_threads(8, cores)          # 8 more tours of each of the 4096 sequences
        rounds += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    steps = o.tables()["steps"]
    o1 = orc.Oracle(w["d"], w["n_max"], w["n_seq"], w["seed"])
    t1 = time.perf_counter()
    r1 = 0
    while True:
        o1.run(1)
        r1 += 1
        el1 = time.perf_counter() - t1
        if el1 >= seconds / 3.0:
            break
    steps1 = o1.tables()["steps"]
    return {"value": steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "Algorithm 2 on %d host threads sharing the table: the first %d tours of each of "
                      "the 4096 sequences of the workload from empty tables (%d growth steps) in %.1f s"
                      % (cores, 8 * rounds, steps, el),
            "single_thread": {"value": steps1 / el1, "unit": UNIT, "cores": 1,
                              "sample": "sequential oracle: the first %d tour(s) of each sequence "
                                        "(%d growth steps) in %.1f s" % (r1, steps1, el1)}}


def batched_to_target(target=3e-2, first_tours=16):
    """The batched forms against the plain per-run form at equal target error: 96
    independent runs (d uniform in {2, 3}, n_max log-uniform in [64, 2048],
    sequences log-uniform in [256, 8192]; PCG64 seed 1), each grown until the
    relative standard error of its c_{n_max} is at most `target`.  Every form
    starts each run with `first_tours` tours per sequence from empty tables and
    then gives each run still above its target the tours the 1/tours law of the
    variance predicts (batch.more_tours), until all meet it:
      - persistent: one persistent kernel over all runs per round (a replay of the
        captured graph, then perm_batch_continue for the runs still short);
      - streams: each run's kernel on one of 64 streams, all concurrent;
      - plain: each run alone on the whole GPU, one after another.
    Wall time to the last run meeting its target, device synchronised."""
    import numpy as np
    import torch
    import paper_2002_03000_gb300 as pg
    from paper_2002_03000_gb300 import batch as pb
    runs = pb.mixed_runs(96, seed=1)
    cfgs = [pb.make_config(d, n, N, 1, run_id=i, max_seconds=120.0) for i, (d, n, N) in enumerate(runs)]
    out = {"workload": "96 independent runs: d uniform in {2,3}, n_max log-uniform in [64,2048], "
                       "sequences log-uniform in [256,8192] (PCG64 seed 1), each to rel. SE of c_nmax <= %g"
                       % target, "target": target, "first_tours_per_seq": first_tours}
    forms = {}
    for form in ("persistent", "streams"):
        b = pb.Batch(cfgs, [first_tours] * len(runs), persistent=(form == "persistent"))
        try:
            b.run()                                   # warm-up replay (graph and kernels loaded)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tours, rounds = b.run_to_target(target)
            tb = time.perf_counter() - t0
            rel = [math.sqrt(b.estimates(r)[2][runs[r][1]]) for r in range(len(runs))]
            steps = sum(b.stats(r)["steps"] for r in range(len(runs)))
            forms[form] = {"seconds": tb, "rounds": rounds, "met": int(sum(x <= target for x in rel)),
                           "steps": steps, "steps_per_s": steps / tb, "total_tours_per_seq": int(sum(tours)),
                           "median_rel_se_c_nmax": float(np.median(rel))}
        except Exception as e:                    # report, do not hide
            forms[form] = {"error": str(e)}
        finally:
            b.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps_p, rel_p, tours_p, failed = 0, [], 0, []
    for i, (d, n, N) in enumerate(runs):
        h = pg.Run(d, n, N, 1, run_id=i, max_seconds=120.0)
        try:
            t = first_tours
            h.run(t)
            for _ in range(8):
                extra = pb.more_tours(h.estimates()[2][n], t, target)
                if not extra:
                    break
                h.run(extra)
                t += extra
            rel_p.append(math.sqrt(h.estimates()[2][n]))
            tours_p += t
        except pg.PermError as e:             # a run past its time bound: reported, not hidden
            failed.append({"run": i, "d_nmax_N": [d, n, N], "error": str(e)})
        steps_p += h.stats()["steps"]
        h.close()
    tp = time.perf_counter() - t0
    plain = {"seconds": tp, "met": int(sum(x <= target for x in rel_p)), "steps": steps_p,
             "steps_per_s": steps_p / tp, "total_tours_per_seq": tours_p,
             "median_rel_se_c_nmax": float(np.median(rel_p)) if rel_p else None, "failed": failed}
    out.update({"persistent": forms["persistent"], "streams": forms["streams"], "plain": plain,
                "timing": "wall clock from the first growth launch to the last run meeting its target"})
    for form in ("persistent", "streams"):
        if "seconds" in forms[form]:
            forms[form]["speedup_vs_plain_to_target"] = tp / forms[form]["seconds"]
    return out


def autotuned_run(tours):
    """The autotuner's choice for the benchmark workload (walks per warp, hash size,
    stack ring; calibrated at equal work, outside the timed region), and one complete
    run from empty tables with it, next to one with the default layout."""
    import torch
    import paper_2002_03000_gb300 as pg
    from paper_2002_03000_gb300 import batch as pb
    w = WORKLOAD
    cfg = pb.make_config(w["d"], w["n_max"], w["n_seq"], w["seed"], max_seconds=120.0)
    t0 = time.perf_counter()
    # probes of a quarter of the run: the tuner validates its pick on runs of
    # four times the probe, i.e. on complete runs of this workload
    pb.autotune(cfg, probe_tours=max(1, tours // 4))
    tune_s = time.perf_counter() - t0
    out = {"lanes_per_warp": cfg.lanes_per_warp, "hash_scale": cfg.hash_scale, "stack_ring": cfg.stack_ring,
           "tune_s": tune_s}
    for name, kw in (("default", {}), ("tuned", {"lanes_per_warp": cfg.lanes_per_warp,
                                                  "hash_scale": cfg.hash_scale, "stack_ring": cfg.stack_ring})):
        run = pg.Run(w["d"], w["n_max"], w["n_seq"], w["seed"], max_seconds=120.0, **kw)
        run.run(2)
        best = None
        for _ in range(3):
            run.reset()
            torch.cuda.synchronize()
            t = time.perf_counter()
            run.run(tours)
            el = time.perf_counter() - t
            best = el if best is None or el < best else best
        out[name + "_s_per_run"] = best
        run.close()
    return out


LOG_MU_REF = {2: 0.970081147258, 3: 1.5441609707}     # literature values quoted in Sec. 5


def growth_constants(sq_estimates):
    """log mu_d from the eq. 15 fit (Sec. 5) to one complete run of each benchmark
    workload: the square run just timed and one cubic run (n_max 512, 8192 x 128)."""
    import numpy as np
    import paper_2002_03000_gb300 as pg
    from paper_2002_03000_gb300.analysis import fit_eq15
    out = {}
    lc2, rv2 = sq_estimates
    import torch
    cub = pg.Run(3, 512, 8192, 1, max_seconds=120.0)
    cub.run(128)                      # a warm-up run, then the timed one from empty tables
    cub.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cub.run(128)
    el = time.perf_counter() - t0
    lc3, _, rv3 = cub.estimates()
    steps3 = cub.stats()["steps"]
    cub.close()
    out["cubic_run"] = {"workload": "d=3 n_max=512 8192 sequences x 128 tours, one complete run from empty tables",
                        "seconds": el, "steps": steps3, "steps_per_s": steps3 / el,
                        "rel_se_c_nmax": math.sqrt(rv3[-1]) if rv3[-1] >= 0 else None,
                        "timing": "wall clock around the run, device synchronised on both sides (one run "
                                  "after a warm-up run)"}
    for d, lc, rv in ((2, lc2, rv2), (3, lc3, rv3)):
        f = fit_eq15(lc, rv, n_min=64, n_max=len(lc) - 1)
        g = fit_eq15(lc, rv, n_min=64, n_max=len(lc) - 1, log_mu=LOG_MU_REF[d])
        out["d%d" % d] = {"log_mu": f["log_mu"], "log_mu_err": f["log_mu_err"], "gamma": f["gamma"],
                          "log_mu_literature": LOG_MU_REF[d],
                          "gamma_with_log_mu_fixed": g["gamma"], "fit_range": [64, len(lc) - 2],
                          "workload": "d=2 n_max=512 4096x256" if d == 2 else "d=3 n_max=512 8192x128"}
    return out


def perm_cutoffs_vs_flatperm(tours=32):
    """Original PERM (Sec. 2, fixed cut-offs) against flatPERM on the bench lattice
    (square, n_max 512, 4096 sequences).  Cut-offs from a pilot flatPERM run of 8
    tours per sequence: T_n = 3 W^_n and t_n = W^_n / 3 with W^_n = W_n / M at the
    stored scale; 2 copies, q = 2.  Then `tours` tours per sequence of each from
    empty tables.  Wall time with the device synchronised; relative standard error
    of c_512 from the per-tour variance."""
    import numpy as np
    import torch
    import paper_2002_03000_gb300 as pg
    d, n_max, N = 2, 512, 4096
    out = {"workload": "square lattice, n_max 512, 4096 sequences x %d tours; PERM cut-offs 3x and 1/3x "
                       "W_n/M of a pilot flatPERM run (8 tours/sequence), 2 copies, q = 2" % tours}
    with pg.Run(d, n_max, N, 3, max_seconds=120.0) as pilot:
        pilot.run(8)
        t = pilot.tables()
    w_hat = t["W"] / float(t["M"][0])
    if not np.all(w_hat > 0):
        out["error"] = "pilot run left lengths unsampled"
        return out
    for form in ("flatperm", "perm_cutoffs"):
        with pg.Run(d, n_max, N, 1, max_seconds=120.0) as run:
            if form == "perm_cutoffs":
                run.set_cutoffs(3.0 * w_hat, w_hat / 3.0, 2, 2.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run.run(tours)
            sec = time.perf_counter() - t0
            lc, S, rv = run.estimates()
            st = run.stats()
        out[form] = {"seconds": sec, "steps": st["steps"], "steps_per_s": st["steps"] / sec,
                     "log_c_nmax": float(lc[n_max]),
                     "rel_se_c_nmax": float(math.sqrt(rv[n_max])) if rv[n_max] > 0 else None,
                     "samples_at_nmax": float(S[n_max])}
    return out


def alg1_vs_alg2():
    """Sec. 4's comparison on the exact-count lattice (square, n_max 16, 12
    sequences): T_16, the mean |log c_n(exact) - log c_n(estimate)| over n = 1..16,
    for Algorithm 1 (private tables, estimates averaged) and Algorithm 2 (one shared
    table), at equal tours per sequence."""
    import numpy as np
    import paper_2002_03000_gb300 as pg
    from paper_2002_03000_gb300.analysis import t_m
    exact = np.log(np.array(EXACT_C_SQUARE, dtype=float))
    rows = []
    for tours in (1, 10, 100, 1000, 10000):
        row = {"tours_per_seq": tours}
        for name, alg in (("alg1", pg.PERM_ALG1), ("alg2", pg.PERM_ALG2)):
            vals = []
            for rep in range(4):
                run = pg.Run(2, 16, 12, 100 + rep, alg=alg, max_seconds=60.0)
                run.run(tours)
                lc = run.estimates()[0]
                run.close()
                vals.append(t_m(lc, exact))
            m = float(np.mean(vals))
            row[name] = m if math.isfinite(m) else None   # a length no sequence reached

        rows.append(row)
    return {"workload": "square lattice, n_max 16, 12 sequences, 4 seeds per point",
            "measure": "T_16 = mean over n=1..16 of |log c_n exact - log c_n estimate|", "rows": rows}


def served_vs_one_at_a_time():
    """Continuous batching against serving one request at a time, on the same
    seeded Poisson stream (150 requests at 50 per second; d uniform in {2, 3};
    n_max log-uniform in [64, 256]; target relative error of c_{n_max} 3e-2 or
    1e-2; 1024 sequences; 4 tours per chunk).  Smaller n_max and looser targets
    than the full request mix keep the session within seconds."""
    from paper_2002_03000_gb300 import serve as ps
    out = {"workload": "150 Poisson requests at 50/s, d in {2,3}, n_max log-uniform [64,256], "
                       "target rel. error of c_nmax in {3e-2, 1e-2}, 1024 sequences, admitted by a "
                       "120 GB device-memory budget"}
    for name, mr in (("continuous", 16), ("one_at_a_time", 1)):
        reqs = ps.poisson_requests(150, 50.0, seed=1, n_max_range=(64, 256), targets=(3e-2, 1e-2), n_seq=1024)
        for r in reqs:
            r.chunk_tours = 4
        srv = ps.Server(ps.GpuEngine(max_ctas=-1 if mr > 1 else 0), hbm_budget_bytes=120e9, max_resident=mr)
        t0 = time.perf_counter()
        done = srv.serve(reqs)
        el = time.perf_counter() - t0
        sm = ps.Server.summary(done, el)
        sm.update({"max_resident": mr, "peak_resident": srv.peak_resident, "wall_s": el})
        out[name] = sm
    return out


REFERENCE_TOURS = 64


def run_reference(args):
    """The oracle on the host cores: each step is a bounded sample of the workload,
    the first REFERENCE_TOURS tours of each of its 4096 sequences from empty tables,
    grown by Algorithm 2 on every host core (threads sharing the table, as the
    paper ran it).  Steps per tour are reported beside the GPU arm's."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as orc
    w = WORKLOAD
    cores = host_cores()
    tot_steps, tot_t, tot_tours = 0, 0.0, 0
    for it in range(args.warmup + args.steps):
        o = orc.Oracle(w["d"], w["n_max"], w["n_seq"], w["seed"], run=it)
        t0 = time.perf_counter()
        o.run_threads(REFERENCE_TOURS, cores)
        el = time.perf_counter() - t0
        if it >= args.warmup:
            tot_steps += o.tables()["steps"]
            tot_t += el
            tot_tours += REFERENCE_TOURS * w["n_seq"]
    val = tot_steps / tot_t
    sample = ("each step: the first %d tours of each of the 4096 sequences from empty tables, "
              "Algorithm 2 on %d host threads sharing the table" % (REFERENCE_TOURS, cores))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (the lattice is the input)",
            "config": {"workload": WORKLOAD_NAME, "d": w["d"], "n_max": w["n_max"],
                       "sequences": w["n_seq"], "tours_per_seq": REFERENCE_TOURS, "seed": w["seed"],
                       "steps_per_tour": tot_steps / tot_tours, "cache": "host CPU",
                       "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_to_target(run, cap_s):
    """Time to a target error, measured on the GPU:
    - the benchmark workload (square, n_max 512, 4096 sequences), one run from empty
      tables continued in chunks of 256 tours per sequence until the relative
      standard error of c_512 (per-tour variance) is at most 1e-3, or `cap_s`; the
      1e-4 time of the metric is extrapolated from it (error ~ 1/sqrt(tours)) and
      labelled so;
    - the exact-count workload (square, n_max 16, 12 sequences), one run continued
      in chunks of 2e4 tours per sequence until the true error
      max_n |c_n(estimate)/c_n - 1| over n <= 16 (exact c_n) is at most 1e-4, or
      `cap_s`.
    Wall clock, each chunk waited for (the estimates are read after every chunk)."""
    import numpy as np
    import torch
    import paper_2002_03000_gb300 as pg
    from paper_2002_03000_gb300 import _native as nat
    w = WORKLOAD
    out = {}
    run.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rel, chunks = float("inf"), 0
    while time.perf_counter() - t0 < cap_s:
        nat.perm_run(run.h, w["tours"])
        chunks += 1
        rv = nat.perm_estimates(run.h, w["n_max"])[2]
        rel = math.sqrt(rv[w["n_max"]])
        if rel <= 1e-3:
            break
    el = time.perf_counter() - t0
    out["bench_workload_rel_se_1e-3"] = {
        "workload": WORKLOAD_NAME + ", continued", "target": "rel. SE of c_512 <= 1e-3",
        "reached": rel <= 1e-3, "seconds": el, "rel_se_at_end": rel,
        "tours_per_seq": chunks * w["tours"], "cap_s": cap_s, "kind": "measured"}
    out["bench_workload_rel_se_1e-4"] = {
        "target": "rel. SE of c_512 <= 1e-4", "seconds": el * (rel / 1e-4) ** 2,
        "kind": "extrapolated from the measured run above (standard error ~ 1/sqrt(tours))"}
    exact = np.array(EXACT_C_SQUARE, dtype=float)
    r1 = pg.Run(2, 16, 12, 1, max_seconds=600.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    err, chunks, trail = float("inf"), 0, []
    while time.perf_counter() - t0 < cap_s:
        r1.run(20000)
        chunks += 1
        lc = r1.estimates()[0]
        err = float(np.max(np.abs(np.exp(lc[:17] - np.log(exact)) - 1.0)))
        trail.append(err)
        if err <= 1e-4:
            break
    el = time.perf_counter() - t0
    st = r1.stats()
    r1.close()
    out["exact_count_workload_true_error_1e-4"] = {
        "workload": "plain flatPERM, d=2, n_max=16, 12 interacting sequences, chunks of 2e4 tours "
                    "per sequence, seed 1",
        "target": "max over n <= 16 of |c_n(estimate)/c_n(exact) - 1| <= 1e-4",
        "reached": err <= 1e-4, "seconds": el, "error_at_end": err, "cap_s": cap_s,
        "tours_per_seq": chunks * 20000, "steps": st["steps"], "steps_per_s": st["steps"] / el,
        "error_after_each_chunk": trail[:8] + (["..."] if len(trail) > 9 else []) + trail[-1:],
        "kind": "measured" if err <= 1e-4 else "not reached within the cap"}
    return out


LOG_C10000_PAPER = 9704.14   # Sec. 4, eq. 8: log c_10000 on the square lattice (1.6e9 iterations)


def long_walks(cap_s=60.0):
    """Sec. 4's long walks with Table 2's setup: square lattice, n_max = 10^4, 12
    interacting sequences (Algorithm 2, snapshot thresholds, walks in the global
    arena), from empty tables, one tour of every sequence per launch until
    `cap_s` seconds (each launch bounded by that too).  Reports what is reached:
    tours finished, growth steps, the longest length sampled, and log c_10000 with
    its standard error against the paper's 9704.14 once n = 10^4 is sampled."""
    import numpy as np
    import paper_2002_03000_gb300 as pg
    n_max, N = 10000, 12
    out = {"workload": "square lattice, n_max 10^4, 12 interacting sequences, from empty tables; "
                       "launches of 1, 2, 4, ... up to 16 tours per sequence", "cap_s": cap_s,
           "log_c10000_paper": LOG_C10000_PAPER, "launches": []}
    # the 12 sequences' tours grow on 12 walks, and helper walks (one walk per SM in
    # all) grow their waiting copies: the start-up trees of reading 20 spread over
    # the device while at most 12 tours are in flight, as with the paper's threads
    helpers = max(0, sm_count() - N)
    run = pg.Run(2, n_max, N, 1, max_seconds=cap_s, helper_walks=helpers)
    out["helper_walks"] = helpers
    t0 = time.perf_counter()
    status, chunk = 0, 1
    while time.perf_counter() - t0 < cap_s:
        t1 = time.perf_counter()
        try:
            run.run(chunk)
        except pg.PermError as e:
            status = e.code
        chunk = min(2 * chunk, 16)
        st = run.stats()
        S = run.tables()["S"]
        reached = int(np.max(np.nonzero(S)[0])) if np.any(S > 0) else 0
        if len(out["launches"]) < 12:
            out["launches"].append({"seconds": time.perf_counter() - t1, "tours_finished": st["tours_finished"],
                                    "steps": st["steps"], "longest_length": reached, "status": st["status"]})
        if status != 0 or st["status"] != 0:
            break
    lc, S, rv = run.estimates()
    st = run.stats()
    run.close()
    wm = {1: "shared memory (one walk per CTA beside the 80 KB snapshot table)", 2: "global arena"}
    reached = int(np.max(np.nonzero(S)[0])) if np.any(S > 0) else 0
    out.update({"seconds": time.perf_counter() - t0, "tours_finished": st["tours_finished"],
                "steps": st["steps"], "longest_length": reached,
                "stopped_by": "time bound of a launch (PERM_ETIMEOUT)" if status or st["status"] else
                              ("cap" if reached < n_max else "n_max reached"),
                "walk_memory": wm.get(st["walk_memory"], str(st["walk_memory"]))})
    if reached >= n_max and math.isfinite(lc[n_max]):
        out["log_c10000"] = float(lc[n_max])
        out["log_c10000_se"] = float(math.sqrt(rv[n_max])) if math.isfinite(rv[n_max]) else None
    else:
        out["log_c_longest"] = float(lc[reached]) if reached > 0 else None
    return out


def table2_long_walks(cap_s=300.0):
    """Sec. 4, Table 2's setup: square lattice, n_max = 10^4, 12 sequences, no helper
    walks (12 walks, as the paper's 12 threads), from empty tables; log c_10000 after
    12 x 1, 12 x 10, 12 x 100 and 12 x 1000 walks (cumulative tours per sequence) for
    Algorithm 2 (one shared table) and Algorithm 1 (private tables: the arithmetic
    combination of Sec. 3 and the geometric one of Sec. 4), each algorithm stopped
    once `cap_s` seconds have passed.  Opt-in (--table2): the Algorithm-1 leg takes
    minutes."""
    import paper_2002_03000_gb300 as pg
    from paper_2002_03000_gb300.analysis import alg1_combine
    paper = {"alg1": {1: 9273.79, 10: 9658.79, 100: 9692.63, 1000: 9703.54},
             "alg2": {1: 9652.09, 10: 9697.79, 100: 9703.23, 1000: 9704.04}}
    out = {"workload": "square lattice, n_max 10^4, 12 sequences, seed 1, no helper walks", "cap_s": cap_s}
    for name, alg in (("alg2", pg.PERM_ALG2), ("alg1", pg.PERM_ALG1)):
        rows = []
        run = pg.Run(2, 10000, 12, 1, alg=alg, max_seconds=max(cap_s, 60.0))
        done, t_all = 0, time.perf_counter()
        for target in (1, 10, 100, 1000):
            if time.perf_counter() - t_all > cap_s:
                break
            t0 = time.perf_counter()
            try:
                run.run(target - done)
            except pg.PermError as e:
                rows.append({"walks_per_seq": target, "error": str(e), "seconds": time.perf_counter() - t0})
                break
            done = target
            lc = run.estimates()[0]
            v = float(lc[10000])
            row = {"walks_per_seq": target, "seconds": time.perf_counter() - t0,
                   "log_c10000": v if math.isfinite(v) else None, "paper": paper[name][target]}
            if alg == pg.PERM_ALG1:
                gv = float(alg1_combine(run.tables(), 2, mode="geometric")[10000])
                row["log_c10000_geometric"] = gv if math.isfinite(gv) else None
            rows.append(row)
        run.close()
        out[name] = rows
    return out


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    from paper_2002_03000_gb300 import build as pbuild
    if rank == 0 or world == 1:
        pbuild.build()
    if world > 1:
        torch.distributed.barrier()
    import numpy as np
    import paper_2002_03000_gb300 as pg
    from paper_2002_03000_gb300 import _native as nat

    w = WORKLOAD
    stream = torch.cuda.Stream()
    run = pg.Run(w["d"], w["n_max"], w["n_seq"], w["seed"], run_id=rank)
    run.set_stream(stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step():
        run.reset()
        nat.perm_run(run.h, w["tours"])

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    st0 = run.stats()

    # ---- device-timed region: K complete runs, L2 flushed between them ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    steps_total, copies_total = 0, 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            torch.cuda.current_stream().synchronize()
            with torch.cuda.stream(stream):
                ev[i][0].record(stream)
                run.reset()
                kev[i][0].record(stream)
                nat.perm_run(run.h, w["tours"])
                kev[i][1].record(stream)
                ev[i][1].record(stream)
            stream.synchronize()
            s = run.stats()
            if s["status"] != 0:
                raise RuntimeError("run failed: %s" % nat.strerror(s["status"]))
            steps_total += s["steps"]
            copies_total += s["copies"]
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    t_dev = sum(step_ms) / 1000.0
    # max over ranks of the device time; sum of steps over ranks
    from paper_2002_03000_gb300 import replicas
    t_dev, steps_all = replicas.reduce_timing(t_dev, steps_total, device="cuda")
    value = steps_all / t_dev

    # ---- end to end through the C ABI, host buffers: run + estimates to host ----
    L = w["n_max"] + 1
    lc, S, rv = np.empty(L), np.empty(L), np.empty(L)
    e2e_steps = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        nat.perm_reset(run.h)
        nat.perm_run(run.h, w["tours"])
        lc, S, rv = nat.perm_estimates(run.h, w["n_max"])
        e2e_steps += run.stats()["steps"]
    e2e_t = time.perf_counter() - t0
    e2e_t, e2e_steps = replicas.reduce_timing(e2e_t, e2e_steps, device="cuda")
    e2e_value = e2e_steps / e2e_t
    # the replicas' last runs pooled into one estimate (sum W_n / sum M)
    pooled = replicas.estimates(replicas.pool_tables(run.tables(), device="cuda"), w["d"])
    d2h = 3 * L * 8 + 4 + 8 * 3 + 8   # W_n, S_n, Q_n tables, status, counters, M

    # ---- time to target error, measured ----
    ttt = None
    if rank == 0 and not args.skip_time_to_target:
        ttt = time_to_target(run, args.target_cap_s)

    f = copies_total / max(steps_total, 1)
    B = bytes_per_step(w["d"], f)
    avg_kern_s = sum(kern_ms) / len(kern_ms) / 1000.0
    steps_per_launch = steps_total / args.steps
    peak, peak_kind = measured_peaks()
    traffic, inst_per_step, traffic_src = measured_counters()
    achieved = B * steps_per_launch / avg_kern_s / 1e9
    clk = clocks.summary()
    issue = None
    if inst_per_step is not None and clk.get("sm_mhz"):
        # warp instructions issued per second against one per scheduler per cycle
        ach = inst_per_step * steps_per_launch / avg_kern_s
        pk = 4.0 * sm_count() * clk["sm_mhz"] * 1e6
        issue = {"achieved": ach, "peak": pk, "unit": "warp instructions/s", "frac": ach / pk,
                 "inst_per_step": inst_per_step, "source": traffic_src,
                 "peak_basis": "4 schedulers x %d SMs x median sampled SM clock" % sm_count()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_dev / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (the lattice is the input)",
        "config": {"workload": WORKLOAD_NAME, "d": w["d"], "n_max": w["n_max"],
                   "sequences": w["n_seq"], "tours_per_seq": w["tours"], "seed": w["seed"],
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "flushed between timed steps (%d MiB write)" % (L2_FLUSH_BYTES >> 20),
                   "step": "one complete run from empty tables"},
        "gpu_launches": 2 * args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_source": traffic_src,
                     "peak_source": peak_kind, "bytes_per_step": B, "copies_per_step": f,
                     "kernel_ms": avg_kern_s * 1000.0,
                     "steps_per_launch": steps_per_launch},
        "issue_roofline": issue,
        "clocks": clk,
        "wall_s_timed": wall,
        "time_to_target": ttt,
        "estimates": {"log_c_nmax": float(lc[w["n_max"]]), "rel_se_c_nmax": float(math.sqrt(rv[w["n_max"]])),
                      "log_c_nmax_over_nmax": float(lc[w["n_max"]] / w["n_max"])},
    }
    if world > 1:
        plc, _, prv = pooled
        line["pooled_estimates"] = {"replicas": world, "log_c_nmax": float(plc[w["n_max"]]),
                                    "rel_se_c_nmax": float(math.sqrt(prv[w["n_max"]])),
                                    "note": "the replicas' last end-to-end runs pooled: sum W_n / sum M"}
    if world == 1 and not args.skip_systems:
        line["growth_constant"] = growth_constants((lc, rv))
        line["alg1_vs_alg2"] = alg1_vs_alg2()
        line["perm_cutoffs"] = perm_cutoffs_vs_flatperm()
        line["long_walks"] = long_walks(args.long_cap_s)
        if args.table2:
            line["table2"] = table2_long_walks(args.table2_cap_s)
        line["autotune"] = autotuned_run(w["tours"])
        line["batched"] = batched_to_target(args.batch_target)
        line["batched"]["stand_in"] = ("stated config: each of the 96 runs to rel. SE of c_nmax <= 1e-3; "
                                       "here: each run to %g (1e-3 needs about 1000 times the tours, "
                                       "~10^4 GPU-s for the mix)" % args.batch_target)
        line["served"] = served_vs_one_at_a_time()
        line["served"]["stand_in"] = ("stated config: n_max log-uniform in [64,1024], targets 1e-3/1e-4, "
                                      "60 s of arrivals; here: 150 requests, n_max in [64,256], targets "
                                      "3e-2/1e-2 (the stated mix needs ~1e2-1e4 GPU-s per request)")
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line), flush=True)
    run.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-time-to-target", action="store_true")
    ap.add_argument("--target-cap-s", type=float, default=60.0)
    ap.add_argument("--skip-systems", action="store_true")
    ap.add_argument("--batch-target", type=float, default=3e-2)
    ap.add_argument("--long-cap-s", type=float, default=30.0)
    ap.add_argument("--table2", action="store_true",
                    help="also run Table 2's setup (n_max 10^4, 12 sequences) for both algorithms (minutes)")
    ap.add_argument("--table2-cap-s", type=float, default=300.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
