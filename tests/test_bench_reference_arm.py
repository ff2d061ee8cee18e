"""The benchmark's reference arm (the oracle timed on the host) keeps its JSON
contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "config", "dtype"):
        assert key in rec, key
    assert rec["value"] > 0 and rec["unit"] == "steps/s"
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == rec["value"] and cb["sample"]
    assert rec["e2e"] == {"value": rec["value"], "unit": rec["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def test_kernel_hash_ignores_comments_only():
    """The hash that keeps the measured DRAM traffic tied to the kernel it was
    measured on changes with the code and not with comments or spacing."""
    sys.path.insert(0, ROOT)
    import bench
    a = "int f(int x) {  // one\n  return x + 1; /* two\n lines */ }\n"
    b = "int f(int x) {\n  return x + 1;   }  // other words\n"
    c = "int f(int x) { return x + 2; }\n"
    assert bench.kernel_sources_sha256([a]) == bench.kernel_sources_sha256([b])
    assert bench.kernel_sources_sha256([a]) != bench.kernel_sources_sha256([c])
