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


def test_traffic_guard_ignores_comments_only():
    """The bench reports the scoring kernel's DRAM traffic only while the
    kernel sources match the ncu capture; the guard's hash leaves comments
    out, so a comment edit keeps it and a code edit voids it."""
    import shutil
    import tempfile
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_2112_07552_gb300", "csrc")
    with tempfile.TemporaryDirectory() as td:
        for f in bench.SCORE_TC_SOURCES:
            shutil.copy(os.path.join(src, f), td)
        h0 = bench.score_tc_src_hash(td)
        assert h0 == bench.score_tc_src_hash()
        p = os.path.join(td, "score_tc.cu")
        with open(p, "a") as fh:
            fh.write("\n// a comment\n/* another\n   comment */\n")
        assert bench.score_tc_src_hash(td) == h0
        with open(p, "a") as fh:
            fh.write("static const int sj_probe_constant = 1;\n")
        assert bench.score_tc_src_hash(td) != h0
    # with a matching hash the traffic scales with the pair-scores
    tr, how = bench.score_tc_traffic(1e12)
    if bench.SCORE_TC_CAPTURE["src_hash"] == bench.score_tc_src_hash():
        assert tr is not None and abs(tr / bench.score_tc_traffic(2e12)[0] - 0.5) < 1e-12, how
    else:
        assert tr is None
