"""The bench's reference arm (the oracle timed on the host) keeps its output
contract: one JSON line with the metric, value, config and the baseline
description, on CPU and in a few seconds at a small shape."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    r = run_bench("--impl", "reference", "--shape", "600,900", "--steps", "1", "--warmup", "1",
                  "--cpu-seconds", "1")
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in r, key
    assert r["impl"] == "reference" and r["metric"] == "pair-scores/s"
    assert r["value"] > 0 and r["higher_is_better"] is True
    assert r["config"]["nA"] == 600 and r["config"]["nB"] == 900
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"]
    assert r["e2e"]["h2d_bytes_per_step"] == 0 and r["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_workloads_say_unavailable():
    r = run_bench("--impl", "reference", "--workload", "infonce")
    assert r["impl"] == "reference" and "unavailable" in r
