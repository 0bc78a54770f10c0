#!/usr/bin/env python3
"""Benchmark of the GB300 similarity join (one JSON line on rank 0).

Workload (the join the throughput figure is quoted on): BF16 scoring with
exact FP32 rescoring, |A| = |B| = 1,000,000, d = 768, clustered synthetic
embeddings (100,000 centres, sigma = 0.1 total noise, 5% near-duplicate pairs
with sigma = 0.02), top-k with k = 20 AND threshold tau = 0.85 from one fused
scoring pass, seed 0.  A step is one full join call (validation, BF16
packing, tensor-core scoring with the fused filter, Dot2/exact rescoring,
ordering, outputs).  Inputs (6.1 GB) exceed L2 (126 MB), so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): weak scaling, each rank joins its own 1M-row A shard
against the replicated B; no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "bf16_similarity_join_1Mx1M_d768_k20_tau0.85",
    "nA": 1_000_000, "nB": 1_000_000, "d": 768, "clusters": 100_000, "sigma": 0.1,
    "near_dup_frac": 0.05, "near_dup_sigma": 0.02, "k": 20, "tau": 0.85, "seed": 0,
    "prec": "bf16",
}
SMALL = dict(WORKLOAD, workload="bf16_similarity_join_65536x65536_d768_k20_tau0.85",
             nA=65536, nB=65536, clusters=6554)
# The 10M x 1M top-k join over Zipf(1.1) cluster sizes (50,000 clusters,
# d = 256, k = 50, no threshold).  Scored with the BF16 hi/lo split: on this
# data the proven margin of E4M3 (~0.1) makes an exact top-k non-selective and
# that of BF16 (~4e-3) still leaves most rows' candidate bands over the list
# capacity; the FP8 error and margin are measured on a sample of rows and
# reported beside the line.
ZIPF = {"workload": "topk_join_10Mx1M_d256_k50_zipf1.1", "nA": 10_000_000, "nB": 1_000_000,
        "d": 256, "clusters": 50_000, "sigma": 0.1, "zipf_s": 1.1, "near_dup_frac": 0.0,
        "near_dup_sigma": 0.0, "k": 50, "tau": None, "seed": 0, "prec": "bf16x3"}
METRIC = "pair-scores/s"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of score_tc_kernel
# per pair-score, from one ncu capture of the one-wave join (19,456 x 262,144,
# d = 768, k = 20, tau = 0.85: 152 row blocks, each sweeping all columns), and
# a hash of the scoring kernel's sources (comments left out) at that capture.  A full launch's
# traffic is this figure times its pair-scores (DRAM bytes grow with the
# waves of row blocks, each re-reading B); the bench reports null when the
# kernel sources no longer match the capture.
SCORE_TC_CAPTURE = {"bytes_per_pair_score": (912868864 + 157973504) / (19456 * 262144),
                    "src_hash": "551db639a37dd57d",
                    "shape": "19456x262144 d=768 k=20 tau=0.85"}
SCORE_TC_SOURCES = ("score_tc.cu", "epilogue.cuh", "tc_common.cuh", "sj_device.cuh")


def strip_comments(src):
    """C++ source without // and /* */ comments or blank lines (string
    literals in these files hold no comment markers)."""
    import re
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def score_tc_src_hash(root=None):
    """Hash of the scoring kernel's sources, comments left out (a comment
    edit does not change the kernel the capture measured)."""
    import hashlib
    h = hashlib.sha256()
    for f in SCORE_TC_SOURCES:
        with open(os.path.join(root or os.path.join(ROOT, "paper_2112_07552_gb300", "csrc"), f),
                  encoding="utf-8") as fh:
            h.update(strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def score_tc_traffic(pair_scores):
    """(traffic bytes of one launch or None, source string)."""
    cap = SCORE_TC_CAPTURE
    if cap["bytes_per_pair_score"] is None:
        return None, "no ncu capture of this kernel"
    if cap["src_hash"] != score_tc_src_hash():
        return None, "kernel changed since the ncu capture (%s)" % cap["shape"]
    return (cap["bytes_per_pair_score"] * pair_scores,
            "ncu capture of %s scaled by pair-scores" % cap["shape"])


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--small", action="store_true", help="65,536 x 65,536 variant (debug)")
    p.add_argument("--shape", default=None,
                   help="nA,nB override of the workload sizes (profiling runs)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--prec", choices=["bf16", "bf16x3", "fp8", "fp32"], default=None,
                   help="scoring precision override (join and zipf workloads); fp32 is "
                        "the CUDA-core comparison form at the same exactness")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--parity-rows", type=int, default=2000,
                   help="zipf workload: cluster-stratified rows checked against the oracle")
    p.add_argument("--no-sub", action="store_true",
                   help="headline only: skip the FP32 form and the other workloads' sub-results")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--workload", choices=["join", "infonce", "batch", "fp8", "zipf",
                                          "relational"],
                   default="join",
                   help="join: the headline similarity join; infonce: the contrastive "
                        "join (65,536 pairs, d = 768, T = 0.05) forward + backward; batch: "
                        "4,096 uneven joins (sizes log-uniform in [100, 50,000] per side, "
                        "d = 384, k = 10, tau = 0.8) in one sj_batch call; fp8: the "
                        "threshold join of the headline data scored in FP8 E4M3 (and in BF16 "
                        "for comparison); zipf: the 10M x 1M top-50 join, d = 256, over "
                        "Zipf(1.1) cluster sizes")
    return p.parse_args()


def make_data(w, rank):
    """(A, B, near-duplicate pairs (i of A, j of B) or None)."""
    from paper_2112_07552_gb300 import datagen
    C = datagen.centres(w["clusters"], w["d"], w["seed"])
    zs = w.get("zipf_s")
    A = datagen.clustered(w["nA"], w["d"], w["clusters"], w["sigma"], w["seed"],
                          stream=0 if rank == 0 else 100 + rank, zipf_s=zs, C=C)
    B = datagen.clustered(w["nB"], w["d"], w["clusters"], w["sigma"], w["seed"], stream=1,
                          zipf_s=zs, C=C)
    if not w["near_dup_frac"]:
        return A, B, None
    A0 = A if rank == 0 else datagen.clustered(w["nA"], w["d"], w["clusters"], w["sigma"],
                                                w["seed"], stream=0, C=C)
    dups = datagen.add_near_duplicates(A0, B, w["near_dup_frac"], w["near_dup_sigma"],
                                       w["seed"])
    return A, B, dups


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(w, A, B, budget_s, gpu_out=None, dups=None):
    """Oracle on a bounded sample of left rows (all of B); returns a dict.
    With near-duplicate pairs given, half the sample is rows that have one."""
    import oracle
    rng = np.random.default_rng(1234)
    rows = rng.choice(w["nA"], size=min(w["nA"], max(2, oracle.num_threads())), replace=False)
    thr = w["tau"] is not None
    t0 = time.perf_counter()
    oracle.topk(A, B, w["k"], rows=rows)
    if thr:
        oracle.threshold(A, B, w["tau"], rows=rows, want_s64=False)
    per_row = (time.perf_counter() - t0) / len(rows)
    n = int(max(2, min(4096, w["nA"], budget_s / max(per_row, 1e-9))))
    n_dup = 0
    if dups is not None and len(dups):
        src = np.unique(dups[:, 0])
        n_dup = min(len(src), n // 2)
        dup_rows = rng.choice(src, size=n_dup, replace=False)
        rest = np.setdiff1d(np.arange(w["nA"]), dup_rows)
        rows = np.sort(np.concatenate(
            [dup_rows, rng.choice(rest, size=min(n - n_dup, len(rest)), replace=False)]))
    else:
        rows = np.sort(rng.choice(w["nA"], size=min(n, w["nA"]), replace=False))
    n = len(rows)
    t0 = time.perf_counter()
    idx, s32, _ = oracle.topk(A, B, w["k"], rows=rows)
    if thr:
        ti, tj, ts, _ = oracle.threshold(A, B, w["tau"], rows=rows, want_s64=False)
    dt = time.perf_counter() - t0
    res = {"value": n * w["nB"] / dt, "unit": METRIC, "cores": oracle.num_threads(),
           "kind": "oracle",
           "sample": "%d left rows (%d with a near duplicate, the rest random) x all %d "
                     "right rows (top-%d%s), %.1f s"
                     % (n, n_dup, w["nB"], w["k"], " + tau=%g" % w["tau"] if thr else "", dt)}
    if gpu_out is not None:
        gidx, gsc, gpairs = gpu_out
        ok = bool(np.array_equal(gidx[rows], idx)
                  and np.array_equal(gsc[rows].view(np.uint32), s32.view(np.uint32)))
        if thr:
            sel = np.isin(gpairs[0], rows)
            ok = ok and np.array_equal(gpairs[0][sel], ti) and np.array_equal(gpairs[1][sel], tj) \
                and np.array_equal(gpairs[2][sel].view(np.uint32), ts.view(np.uint32))
        res["parity_rows_exact"] = ok
    return res


def join_config(w, world):
    """The config object of a join line (both arms)."""
    in_gb = (w["nA"] + w["nB"]) * w["d"] * 4 / 1e9
    return {"workload": w["workload"], "nA": w["nA"], "nB": w["nB"], "d": w["d"], "k": w["k"],
            "tau": w["tau"], "clusters": w["clusters"], "zipf_s": w.get("zipf_s"),
            "seed": w["seed"],
            "l2": ("inputs %.1f GB > L2, no flush" % in_gb) if in_gb > 0.13
                  else "inputs %.3f GB (small debug shape, fits in L2)" % in_gb,
            "parallelism": "dp%d" % world}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    A, B, dups = make_data(w, 0)
    import oracle
    oracle.build()
    vals = []
    last = None
    for s in range(args.warmup + args.steps):
        r = cpu_baseline(w, A, B, max(1.0, args.cpu_seconds / 3), dups=dups)
        if s >= args.warmup:
            vals.append(r["value"])
            last = r
    v = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": join_config(w, 1),
           "cpu_baseline": {"value": v, "unit": METRIC, "cores": last["cores"],
                            "kind": "oracle", "sample": last["sample"]},
           "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


INFONCE = {"workload": "infonce_fwd_bwd_65536_d768_T0.05", "n": 65536, "d": 768,
           "T": 0.05, "clusters": 100_000, "sigma_pair": 0.02, "seed": 0}


def infonce_cpu_baseline(A, B, T, budget_s):
    """The oracle's row logsumexp + dA row on a bounded sample of rows (all
    columns each), sized from a 16-row probe to about budget_s seconds."""
    import torch

    import oracle
    n = A.shape[0]
    ab = torch.from_numpy(A).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    bb = torch.from_numpy(B).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    probe = np.arange(min(n, max(2, oracle.num_threads())))
    t0 = time.perf_counter()
    oracle.infonce_rows(ab, bb, T, probe)
    per_row = (time.perf_counter() - t0) / len(probe)
    m = int(max(len(probe), min(n, 4096, budget_s / max(per_row, 1e-9))))
    rows = np.sort(np.random.default_rng(5).choice(n, size=m, replace=False))
    t0 = time.perf_counter()
    oracle.infonce_rows(ab, bb, T, rows)
    dt = time.perf_counter() - t0
    return {"value": len(rows) * n / dt, "unit": METRIC, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "%d random rows: row logsumexp + dA row over all %d columns, %.1f s"
                      % (len(rows), n, dt)}


def run_infonce(args, steps=None, warmup=None, cpu_seconds=None, e2e=True):
    """Contrastive join: one step = forward (loss, lse) + backward (dA, dB).
    Returns the line (a dict)."""
    steps = steps or args.steps
    warmup = warmup or args.warmup
    cpu_seconds = args.cpu_seconds if cpu_seconds is None else cpu_seconds
    import torch

    from paper_2112_07552_gb300 import _build, datagen, sj
    w = dict(INFONCE)
    if args.shape:
        w["n"] = int(args.shape.split(",")[0])
    n, d, T = w["n"], w["d"], w["T"]
    _build.build()
    A, B = datagen.paired(n, d, w["clusters"], 0.1, w["sigma_pair"], seed=w["seed"])
    dev = torch.device("cuda", 0)
    dA = torch.from_numpy(A).to(dev)
    dB = torch.from_numpy(B).to(dev)
    stream = torch.cuda.current_stream(dev)
    J = sj.SimilarityJoin(d, prec="bf16", device=0, stream=stream)
    g = torch.ones(1, device=dev)

    def step(Ain, Bin):
        loss, lse = J.contrastive_forward(Ain, Bin, T)
        gA, gB = J.contrastive_backward(Ain, Bin, T, lse, g)
        return loss

    for _ in range(warmup):
        step(dA, dB)
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        J.contrastive_forward(dA, dB, T)
    e1.record(stream)
    loss, lse = J.contrastive_forward(dA, dB, T)
    e1b = torch.cuda.Event(enable_timing=True)
    e1b.record(stream)
    for _ in range(steps):
        J.contrastive_backward(dA, dB, T, lse, g)
    e2.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_fwd = e0.elapsed_time(e1) / steps
    ms_bwd = e1b.elapsed_time(e2) / steps
    ms = ms_fwd + ms_bwd
    # e2e: pinned host inputs copied in, loss read back, every step
    e_ms = None
    if e2e:
        hA = torch.from_numpy(A).pin_memory()
        hB = torch.from_numpy(B).pin_memory()
        t0 = time.perf_counter()
        for _ in range(steps):
            xa = hA.to(dev, non_blocking=True)
            xb = hB.to(dev, non_blocking=True)
            float(step(xa, xb).item())
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - t0) * 1e3 / steps
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    flops = 8.0 * n * n * d  # algorithmic: S (2N^2 d) + dA, dB, S-recompute (6N^2 d)
    achieved = flops / (ms / 1e3) / 1e12
    cpu = None
    if not args.no_cpu and cpu_seconds > 0:
        cpu = infonce_cpu_baseline(A, B, T, cpu_seconds)
    out = {
        "metric": METRIC, "value": n * n / (ms / 1e3), "unit": METRIC, "n_gpus": 1,
        "steps": steps, "warmup": warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": w["workload"], "n": n, "d": d, "T": T,
                   "l2": "inputs 0.4 GB > L2, no flush"},
        "stages_ms": {"forward": ms_fwd, "backward": ms_bwd},
        "roofline": {"bound": "tensor", "kernel": "contrastive_kernel", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": src + " bf16_tflops_sustained", "traffic": None,
                     "flops_per_step": flops},
        # forward: two packs, the forward kernel, the merge of its partial row
        # states, the loss reduction; backward: two packs, the dL/dS pass, two
        # GEMMs (K forwards, one more for lse, K backwards in the timed region)
        "gpu_launches": 5 * (steps + 1) + 5 * steps,
        "clocks": clocks,
        "e2e": None if e_ms is None else
               {"value": n * n / (e_ms / 1e3), "unit": METRIC, "ms_per_step": e_ms,
                "h2d_bytes_per_step": int(2 * n * d * 4), "d2h_bytes_per_step": 4},
        "cpu_baseline": cpu,
    }
    J.close()
    return out


BATCH = {"workload": "bf16_batch_4096_jobs_loguniform_100-50000_d384_k10_tau0.8",
         "n_jobs": 4096, "lo": 100, "hi": 50_000, "d": 384, "k": 10, "tau": 0.8,
         "sigma": 0.1, "seed": 0}


def run_batch(args, steps=None, warmup=None, e2e=True):
    """Uneven batch: one step = one sj_batch call over every job (top-k and
    threshold of each job from one scoring pass).  Returns the line."""
    steps = steps or args.steps
    warmup = warmup or args.warmup
    import ctypes

    import torch

    from paper_2112_07552_gb300 import _build, datagen, sj
    w = dict(BATCH)
    if args.shape:
        w["n_jobs"] = int(args.shape.split(",")[0])
        w["workload"] = w["workload"].replace("4096", str(w["n_jobs"]))
    nj, d, k, tau = w["n_jobs"], w["d"], w["k"], w["tau"]
    sa = datagen.log_uniform_sizes(nj, w["lo"], w["hi"], w["seed"], 0)
    sb = datagen.log_uniform_sizes(nj, w["lo"], w["hi"], w["seed"], 1)
    pair_scores = float(np.sum(sa.astype(np.float64) * sb))
    _build.build()
    L = sj.lib()
    dev = torch.device("cuda", 0)
    t_gen = time.perf_counter()
    A, B, ao, bo = datagen.clustered_batch_device(sa, sb, d, w["sigma"], w["seed"], device=dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.current_stream(dev)
    J = sj.SimilarityJoin(d, prec="bf16", device=0, stream=stream)
    # tile widths per right-side size class from the autotuner (untimed)
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        t_tune = time.perf_counter()
        J.autotune(k, os.path.join(td, "tiles.txt"))
        t_tune = time.perf_counter() - t_tune
        widths = {int(r[3]): int(r[4]) for r in
                  (line.split() for line in open(os.path.join(td, "tiles.txt")))}
    caps = 16 * sa + 1024
    po = np.concatenate([[0], np.cumsum(caps)])
    n_out = (sj.I64 * nj)()

    def make_jobs(q0, q1, a_ptr, b_ptr, i_ptr, s_ptr, p_ptr):
        arr = (sj.SjJob * (q1 - q0))()
        for t, q in enumerate(range(q0, q1)):
            arr[t].A = a_ptr + int(ao[q] - ao[q0]) * d * 4
            arr[t].nA = int(sa[q])
            arr[t].B = b_ptr + int(bo[q] - bo[q0]) * d * 4
            arr[t].nB = int(sb[q])
            arr[t].k, arr[t].tau = k, tau
            arr[t].topk_idx = i_ptr + int(ao[q] - ao[q0]) * k * 8
            arr[t].topk_score = s_ptr + int(ao[q] - ao[q0]) * k * 4
            arr[t].pairs = p_ptr + int(po[q] - po[q0]) * 24
            arr[t].capacity = int(caps[q])
            arr[t].n_out = sj.P(ctypes.addressof(n_out) + 8 * q)
        return arr

    idx = torch.empty((int(ao[-1]), k), dtype=torch.int64, device=dev)
    sc = torch.empty((int(ao[-1]), k), dtype=torch.float32, device=dev)
    pairs = torch.empty((int(po[-1]), 3), dtype=torch.int64, device=dev)
    jobs = make_jobs(0, nj, A.data_ptr(), B.data_ptr(), idx.data_ptr(), sc.data_ptr(),
                     pairs.data_ptr())

    def step(arr, n):
        st = sj.SjStats()
        code = L.sj_batch(J.handle, arr, n, ctypes.byref(st))
        if code != sj.SJ_OK:
            raise sj.SJError(code, "sj_batch")
        return st

    for _ in range(warmup):
        step(jobs, nj)
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [step(jobs, nj) for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / steps
    ms_score = statistics.mean(s.ms_score for s in stats)
    n_pairs_all = int(sum(n_out[q] for q in range(nj)))
    padded = float(stats[-1].padded_pair_scores)

    # parity on sampled rows of sampled jobs, and the oracle's time on them
    import oracle
    rng = np.random.default_rng(4321)
    sample_jobs = np.sort(rng.choice(nj, size=min(nj, 12), replace=False))
    ok = True
    cpu_pairs, cpu_t = 0.0, 0.0
    for q in sample_jobs:
        rows = np.sort(rng.choice(int(sa[q]), size=min(int(sa[q]), 24), replace=False))
        Aq = A[int(ao[q]):int(ao[q + 1])][torch.from_numpy(rows).to(dev)].cpu().numpy()
        Bq = B[int(bo[q]):int(bo[q + 1])].cpu().numpy()
        t0 = time.perf_counter()
        wi, ws, _ = oracle.topk(Aq, Bq, k)
        ti, tj, ts, _ = oracle.threshold(Aq, Bq, tau, want_s64=False)
        cpu_t += time.perf_counter() - t0
        cpu_pairs += len(rows) * float(sb[q])
        gi = idx[int(ao[q]):int(ao[q + 1])].cpu().numpy()[rows]
        gs = sc[int(ao[q]):int(ao[q + 1])].cpu().numpy()[rows]
        ok = ok and np.array_equal(gi, wi) and np.array_equal(gs.view(np.uint32), ws.view(np.uint32))
        m = int(n_out[q])
        gp = pairs[int(po[q]):int(po[q]) + m].cpu()
        pi, pj = gp[:, 0].numpy(), gp[:, 1].numpy()
        ps = gp[:, 2:3].contiguous().view(torch.float32)[:, 0].numpy()
        sel = np.isin(pi, rows)
        pos = np.searchsorted(rows, pi[sel])
        ok = ok and np.array_equal(pos, ti) and np.array_equal(pj[sel], tj) \
            and np.array_equal(ps[sel].view(np.uint32), ts.view(np.uint32))
    cpu = {"value": cpu_pairs / cpu_t, "unit": METRIC, "cores": oracle.num_threads(),
           "kind": "oracle",
           "sample": "%d jobs x up to 24 random left rows x all right rows of the job "
                     "(top-%d + tau=%g), %.1f s" % (len(sample_jobs), k, tau, cpu_t),
           "parity_rows_exact": bool(ok)}

    # end to end on the leading jobs holding a quarter of the rows: pinned host
    # inputs and outputs through the same call
    e2e = None
    if e2e and not args.no_e2e:
        rows_tot = np.cumsum(sa + sb)
        qe = int(max(1, np.searchsorted(rows_tot, rows_tot[-1] / 4)))
        hA = A[:int(ao[qe])].cpu().pin_memory()
        hB = B[:int(bo[qe])].cpu().pin_memory()
        del idx, sc, pairs
        torch.cuda.empty_cache()
        hidx = torch.empty((int(ao[qe]), k), dtype=torch.int64).pin_memory()
        hsc = torch.empty((int(ao[qe]), k), dtype=torch.float32).pin_memory()
        hpairs = torch.empty((int(po[qe]), 3), dtype=torch.int64).pin_memory()
        hjobs = make_jobs(0, qe, hA.data_ptr(), hB.data_ptr(), hidx.data_ptr(),
                          hsc.data_ptr(), hpairs.data_ptr())
        step(hjobs, qe)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            step(hjobs, qe)
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - t0) * 1e3 / steps
        sub = float(np.sum(sa[:qe].astype(np.float64) * sb[:qe]))
        e2e = {"value": sub / (e_ms / 1e3), "unit": METRIC, "ms_per_step": e_ms,
               "jobs": qe, "pair_scores_per_step": sub,
               "h2d_bytes_per_step": int((ao[qe] + bo[qe]) * d * 4),
               "d2h_bytes_per_step": int(ao[qe] * k * 12
                                         + sum(int(n_out[q]) for q in range(qe)) * 24)}
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    achieved = 2.0 * pair_scores * d / (ms_score / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": pair_scores / (ms / 1e3), "unit": METRIC, "n_gpus": 1,
        "steps": steps, "warmup": warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": w["workload"], "n_jobs": nj, "rows_A": int(ao[-1]),
                   "rows_B": int(bo[-1]), "pair_scores": pair_scores, "d": d, "k": k,
                   "tau": tau, "seed": w["seed"],
                   "l2": "inputs %.0f GB > L2, no flush" % ((ao[-1] + bo[-1]) * d * 4 / 1e9),
                   "parallelism": "dp1",
                   "tile_widths_by_nB_class": widths, "autotune_s": t_tune},
        "roofline": {"bound": "tensor", "kernel": "score_tc_kernel", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": src + " bf16_tflops_sustained", "traffic": None,
                     "ms_kernel": ms_score, "tile_waste": padded / pair_scores - 1.0},
        "stages_ms": {"prepare": statistics.mean(s.ms_prepare for s in stats),
                      "score": ms_score,
                      "select": statistics.mean(s.ms_select for s in stats)},
        "n_pairs": n_pairs_all,
        "n_rescored": int(stats[-1].n_rescored),
        "n_overflow_rows": int(stats[-1].n_overflow_rows),
        "gpu_launches": int(sum(s.n_launches for s in stats)),
        "generate_s": t_gen,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    J.close()
    return out


def fp8_peak_tflops():
    """Dense FP8 E4M3 tensor peak measured here: torch._scaled_mm (cuBLASLt)
    at 8192^3, best of 5 after 3 warm-ups (burst), or None if unavailable."""
    import torch
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        best = 1e30
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b
        return 2.0 * n ** 3 / (best / 1e3) / 1e12
    except Exception:
        return None


def run_fp8(args, data=None, steps=None, warmup=None):
    """Threshold join of the headline data (1M x 1M, d = 768, tau = 0.85)
    scored in FP8 E4M3 with exact rescoring; the same join in BF16 is timed
    beside it.  (Exact FP8 top-k is not measured: with the rigorous E4M3
    margin the running k-th best stays within 2m of the bulk until a row's
    best matches appear, so every band list overflows into the rescan.)
    `data` = (A, B, dA, dB) reuses the caller's inputs.  Returns the line."""
    steps = steps or args.steps
    warmup = warmup or args.warmup
    import ctypes

    import torch

    from paper_2112_07552_gb300 import _build, sj
    w = dict(WORKLOAD)
    if args.shape:
        nA, nB = (int(x) for x in args.shape.split(","))
        w.update(nA=nA, nB=nB, clusters=max(1, nB // 10))
    nA, nB, d, tau = w["nA"], w["nB"], w["d"], w["tau"]
    _build.build()
    L = sj.lib()
    dev = torch.device("cuda", 0)
    if data is None:
        A, B, _ = make_data(w, 0)
        dA = torch.from_numpy(A).to(dev)
        dB = torch.from_numpy(B).to(dev)
    else:
        A, B, dA, dB = data
    stream = torch.cuda.current_stream(dev)
    cap = 40_000_000
    pairs = torch.empty((cap, 3), dtype=torch.int64, device=dev)
    n_out = sj.I64(0)
    res = {}
    for prec in ("fp8", "bf16"):
        J = sj.SimilarityJoin(d, prec=prec, device=0, stream=stream)
        jb = (sj.SjJob * 1)()
        jb[0].A, jb[0].nA, jb[0].B, jb[0].nB = dA.data_ptr(), nA, dB.data_ptr(), nB
        jb[0].tau, jb[0].pairs, jb[0].capacity = tau, pairs.data_ptr(), cap
        jb[0].n_out = ctypes.cast(ctypes.byref(n_out), sj.P)

        def step():
            st = sj.SjStats()
            code = L.sj_batch(J.handle, jb, 1, ctypes.byref(st))
            if code != sj.SJ_OK:
                raise sj.SJError(code, "sj_batch")
            return st
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        clk = ClockSampler(0)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = [step() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1) / steps
        got = (pairs[:n_out.value, 0].cpu().numpy(), pairs[:n_out.value, 1].cpu().numpy(),
               pairs[:n_out.value, 2:3].contiguous().view(torch.float32)[:, 0].cpu().numpy())
        res[prec] = {"ms": ms, "ms_score": statistics.mean(s.ms_score for s in stats),
                     "ms_select": statistics.mean(s.ms_select for s in stats),
                     "n_pairs": int(n_out.value), "n_candidates": int(stats[-1].n_candidates),
                     "n_exact": int(stats[-1].n_exact), "clocks": clocks, "pairs": got,
                     "launches": int(sum(s.n_launches for s in stats))}
        J.close()
    same = all(np.array_equal(a_, b_) for a_, b_ in zip(res["fp8"]["pairs"], res["bf16"]["pairs"]))
    # parity against the oracle on sampled rows
    import oracle
    rng = np.random.default_rng(99)
    rows = np.sort(rng.choice(nA, size=max(2, oracle.num_threads()), replace=False))
    t0 = time.perf_counter()
    ti, tj, ts, _ = oracle.threshold(A, B, tau, rows=rows, want_s64=False)
    cpu_t = time.perf_counter() - t0
    gi, gj, gs = res["fp8"]["pairs"]
    sel = np.isin(gi, rows)
    ok = bool(np.array_equal(gi[sel], ti) and np.array_equal(gj[sel], tj)
              and np.array_equal(gs[sel].view(np.uint32), ts.view(np.uint32)))
    peaks, src = measured_peaks()
    peak8 = fp8_peak_tflops()
    if peak8:
        peak, peak_source = peak8, "measured here: torch._scaled_mm E4M3 8192^3, best of 5"
    else:
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))) * 2.0
        peak_source = src + " bf16_tflops_sustained x 2 (FP8/BF16 nominal ratio)"
    r8 = res["fp8"]
    achieved = 2.0 * nA * nB * d / (r8["ms_score"] / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": nA * nB / (r8["ms"] / 1e3), "unit": METRIC, "n_gpus": 1,
        "steps": steps, "warmup": warmup, "ms_per_step": r8["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp8_e4m3",
        "data": "synthetic",
        "config": {"workload": "fp8_threshold_join_%dx%d_d%d_tau%g" % (nA, nB, d, tau),
                   "nA": nA, "nB": nB, "d": d, "tau": tau, "clusters": w["clusters"],
                   "seed": w["seed"], "l2": "inputs 6.1 GB > L2, no flush",
                   "parallelism": "dp1"},
        "roofline": {"bound": "tensor", "kernel": "score_tc_kernel<fp8>", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": peak_source, "traffic": None, "ms_kernel": r8["ms_score"]},
        "stages_ms": {"score": r8["ms_score"], "select": r8["ms_select"]},
        "n_pairs": r8["n_pairs"], "n_candidates": r8["n_candidates"], "n_exact": r8["n_exact"],
        "bf16_same_join": {"ms_per_step": res["bf16"]["ms"], "ms_score": res["bf16"]["ms_score"],
                           "value": nA * nB / (res["bf16"]["ms"] / 1e3),
                           "pairs_identical_to_fp8": same},
        "gpu_launches": r8["launches"],
        "clocks": r8["clocks"],
        "e2e": None,
        "cpu_baseline": {"value": len(rows) * nB / cpu_t, "unit": METRIC,
                         "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "%d random left rows x all %d right rows (tau=%g), %.1f s"
                                   % (len(rows), nB, tau, cpu_t),
                         "parity_rows_exact": ok},
    }
    del pairs
    return out


def zipf_parity(w, A, B, gidx, gsc, n_rows=2000):
    """Oracle parity of the top-k on cluster-stratified rows: the clusters are
    ranked by size (Zipf rank), cut into four strata holding a quarter of
    the rows each (the few largest clusters first), and n_rows/4 rows are
    drawn from each, so the dense bands of the big clusters are covered."""
    import oracle
    from paper_2112_07552_gb300 import datagen
    asg = datagen.assignments(w["nA"], w["clusters"], w["seed"], 0, w.get("zipf_s"))
    sizes = np.bincount(asg, minlength=w["clusters"])
    order = np.argsort(-sizes, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    row_rank = rank[asg]
    cum = np.cumsum(sizes[order]) / w["nA"]
    cuts = [int(np.searchsorted(cum, q)) for q in (0.25, 0.5, 0.75)]
    edges = [0] + cuts + [w["clusters"]]
    rng = np.random.default_rng(77)
    rows, strata = [], []
    for t in range(4):
        cand = np.nonzero((row_rank >= edges[t]) & (row_rank < edges[t + 1]))[0]
        take = min(len(cand), n_rows // 4)
        rows.append(rng.choice(cand, size=take, replace=False))
        strata.append({"cluster_ranks": [int(edges[t]), int(edges[t + 1])], "rows": take})
    rows = np.sort(np.concatenate(rows))
    t0 = time.perf_counter()
    idx, s32, _ = oracle.topk(A, B, w["k"], rows=rows)
    dt = time.perf_counter() - t0
    ok = bool(np.array_equal(gidx[rows], idx)
              and np.array_equal(gsc[rows].view(np.uint32), s32.view(np.uint32)))
    return {"rows": int(len(rows)), "strata": strata, "exact": ok, "oracle_seconds": dt,
            "oracle_cores": oracle.num_threads(),
            "oracle_pair_scores_per_s": len(rows) * w["nB"] / dt}


def fp8_error_sample(w, A, B, dB, rows=16):
    """E4M3 scoring error against FP64 on every pair of a row sample: the raw
    E4M3 scores of `rows` rows against all of B (sj_debug_scores) against the
    oracle's FP64 enclosure of each exact score, with the proven margins."""
    import torch

    import oracle
    from paper_2112_07552_gb300 import sj
    sel = np.linspace(0, w["nA"] - 1, rows).astype(np.int64)
    As = np.ascontiguousarray(A[sel])
    dA = torch.from_numpy(As).cuda()
    raw = torch.empty((rows, w["nB"]), dtype=torch.float32, device="cuda")
    marg = torch.empty(rows, dtype=torch.float32, device="cuda")
    with sj.SimilarityJoin(w["d"], prec="fp8", device=0) as J:
        sj._check(sj.lib().sj_debug_scores(J.handle, raw.data_ptr(), marg.data_ptr()),
                  "sj_debug_scores")
        J.topk(dA, dB, w["k"])
    torch.cuda.synchronize()
    lo, hi = oracle.enclose_all(As, B)
    r = raw.cpu().numpy().astype(np.float64)
    m = marg.cpu().numpy().astype(np.float64)
    err = np.maximum(r - lo, hi - r)
    return {"rows": rows, "pairs": int(r.size), "max_abs_err": float(err.max()),
            "mean_abs_err": float(np.abs(r - 0.5 * (lo + hi)).mean()),
            "margin_max": float(m.max()), "max_err_over_margin": float((err / m[:, None]).max())}


def guarded(fn, *a, **kw):
    """A sub-result of the line: its dict, or the error that stopped it."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 -- reported in the line, not fatal
        return {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}


def fp32_same_join(args, w, dA, dB, stream, idx_bf16, sc_bf16, pairs_bf16, value_bf16,
                   rows=16384, steps=3, warmup=1):
    """The plain FP32 CUDA-core form of the headline join at the same
    exactness, on its first `rows` left rows against all of B (a rate does not
    depend on the number of rows): pair-scores/s, the BF16 headline's speed-up
    over it, and whether both emit the same top-k and pairs for those rows."""
    import ctypes

    import torch

    from paper_2112_07552_gb300 import sj
    L = sj.lib()
    nB, d, k, tau = w["nB"], w["d"], w["k"], w["tau"]
    n = min(rows, w["nA"])
    cap = 4_000_000
    idx = torch.empty((n, k), dtype=torch.int64, device=dA.device)
    sc = torch.empty((n, k), dtype=torch.float32, device=dA.device)
    pairs = torch.empty((cap, 3), dtype=torch.int64, device=dA.device)
    n_out = sj.I64(0)
    J = sj.SimilarityJoin(d, prec="fp32", device=dA.device.index, stream=stream)
    jb = (sj.SjJob * 1)()
    jb[0].A, jb[0].nA, jb[0].B, jb[0].nB = dA.data_ptr(), n, dB.data_ptr(), nB
    jb[0].k, jb[0].topk_idx, jb[0].topk_score = k, idx.data_ptr(), sc.data_ptr()
    jb[0].tau, jb[0].pairs, jb[0].capacity = tau, pairs.data_ptr(), cap
    jb[0].n_out = ctypes.cast(ctypes.byref(n_out), sj.P)
    stats = []
    for it in range(warmup + steps):
        st = sj.SjStats()
        code = L.sj_batch(J.handle, jb, 1, ctypes.byref(st))
        if code != sj.SJ_OK:
            raise sj.SJError(code, "sj_batch (fp32)")
        if it >= warmup:
            stats.append(st)
    torch.cuda.synchronize()
    J.close()
    ms = statistics.mean(s.ms_total for s in stats)
    ms_score = statistics.mean(s.ms_score for s in stats)
    v = n * nB / (ms / 1e3)
    m = int(n_out.value)
    gi, gj, gs = pairs_bf16
    sel = gi < n
    same = bool(torch.equal(idx, idx_bf16[:n])
                and torch.equal(sc.view(torch.int32), sc_bf16[:n].view(torch.int32))
                and m == int(sel.sum())
                and np.array_equal(pairs[:m, 0].cpu().numpy(), gi[sel])
                and np.array_equal(pairs[:m, 1].cpu().numpy(), gj[sel])
                and np.array_equal(pairs[:m, 2:3].contiguous().view(torch.float32)[:, 0]
                                   .cpu().numpy().view(np.uint32), gs[sel].view(np.uint32)))
    sms = torch.cuda.get_device_properties(dA.device).multi_processor_count
    return {"rows": n, "value": v, "unit": METRIC, "ms_per_step": ms, "ms_score": ms_score,
            "score_tflops": 2.0 * n * nB * d / (ms_score / 1e3) / 1e12,
            "bf16_speedup": value_bf16 / v, "outputs_identical_to_bf16": same,
            "fp32_lanes_peak_note": "%d SMs x 128 FP32 lanes x 2 flop per clock" % sms}


CONFIG1 = {"workload": "fp32_similarity_join_2000x2000_d256_k10_tau0.8", "nA": 2000,
           "nB": 2000, "d": 256, "clusters": 200, "sigma": 0.1, "near_dup_frac": 0.0,
           "near_dup_sigma": 0.0, "k": 10, "tau": 0.8, "seed": 0}


def run_config1(args, steps=5, warmup=3):
    """The small join (2,000 x 2,000, d = 256, 200 centres, k = 10 and
    tau = 0.8) in the FP32 CUDA-core form and in BF16, each checked in full
    against the oracle (which finishes it in seconds)."""
    import torch

    import oracle
    from paper_2112_07552_gb300 import sj
    w = dict(CONFIG1)
    A, B, _ = make_data(w, 0)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    t0 = time.perf_counter()
    w_idx, w_s, _ = oracle.topk(A, B, w["k"])
    ti, tj, ts, _ = oracle.threshold(A, B, w["tau"], want_s64=False)
    cpu_t = time.perf_counter() - t0
    res = {"config": w, "oracle": {"value": w["nA"] * w["nB"] / cpu_t, "unit": METRIC,
                                   "cores": oracle.num_threads(), "seconds": cpu_t}}
    for prec in ("fp32", "bf16"):
        J = sj.SimilarityJoin(w["d"], prec=prec, device=0)
        for _ in range(warmup):
            out = J.batch([{"A": dA, "B": dB, "k": w["k"], "tau": w["tau"]}])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            out = J.batch([{"A": dA, "B": dB, "k": w["k"], "tau": w["tau"]}])
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / steps
        J.close()
        o = out[0]
        exact = bool(np.array_equal(o["idx"].cpu().numpy(), w_idx)
                     and np.array_equal(o["score"].cpu().numpy().view(np.uint32),
                                        w_s.view(np.uint32))
                     and np.array_equal(o["i"].cpu().numpy(), ti)
                     and np.array_equal(o["j"].cpu().numpy(), tj)
                     and np.array_equal(o["pair_score"].cpu().numpy().view(np.uint32),
                                        ts.view(np.uint32)))
        res[prec] = {"value": w["nA"] * w["nB"] / (ms / 1e3), "unit": METRIC,
                     "ms_per_call": ms, "n_pairs": int(len(o["i"])),
                     "parity_full_exact": exact,
                     "timing": "host wall clock per sj_batch call (launch-latency bound)"}
    return res


def run_relational(args, steps=3, warmup=1):
    """The paper's relational patterns at its entity-matching and
    microbenchmark shapes: blocking of iTunes-Amazon (6,907 x 55,923) on
    Price (12 distinct values, ~32M pairs) and on all six attributes with
    >= 3 equal; Q3/Q4 aggregates over 1M x 1M (ID, Val) tables with 1,000
    distinct IDs.  Wall time per call (host dictionary encoding included),
    results checked against the relational oracle."""
    import torch

    from oracle import relational
    from paper_2112_07552_gb300 import datagen, sj
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "em_blocking_shapes.json")))
    it = g["itunes_amazon"]
    J = sj.SimilarityJoin(8, prec="bf16", device=0)
    res = {}

    def timed(fn):
        for _ in range(warmup):
            out = fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            out = fn()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) / steps

    for name, attrs, m in (("em_blocking_itunes_price", ["Price"], 1),
                           ("em_blocking_itunes_6attr_ge3",
                            ["Price", "Genre", "Time", "Artist", "Copyright", "Album"], 3)):
        ka = np.stack([datagen.keys(it["rows"][0], it["distinct"][a], t, 0)
                       for t, a in enumerate(attrs)], axis=1)
        kb = np.stack([datagen.keys(it["rows"][1], it["distinct"][a], t, 1)
                       for t, a in enumerate(attrs)], axis=1)
        dka, dkb = torch.from_numpy(ka).cuda(), torch.from_numpy(kb).cuda()
        (i, j, sc), t = timed(lambda: J.block(dka, dkb, m, capacity=40_000_000))
        wi, wj, ws = relational.block(ka, kb, m)
        res[name] = {"nA": int(ka.shape[0]), "nB": int(kb.shape[0]), "n_attr": len(attrs),
                     "min_match": m, "n_pairs": int(len(wi)), "seconds_per_call": t,
                     "pair_scores_per_s": ka.shape[0] * kb.shape[0] / t,
                     "pairs_out_per_s": len(wi) / t,
                     "parity_exact": bool(np.array_equal(i.cpu().numpy(), wi)
                                          and np.array_equal(j.cpu().numpy(), wj)
                                          and np.array_equal(sc.cpu().numpy().view(np.uint32),
                                                             ws.view(np.uint32)))}
        del i, j, sc
    rng = np.random.default_rng(11)
    n = 1_000_000
    a_id = rng.integers(0, 1000, size=n).astype(np.int64)
    b_id = rng.integers(0, 1000, size=n).astype(np.int64)
    a_val = rng.integers(-2 ** 31, 2 ** 31, size=n).astype(np.int32)
    b_val = rng.integers(-2 ** 31, 2 ** 31, size=n).astype(np.int32)
    b_g = rng.integers(0, 500, size=n).astype(np.int64)
    d = [torch.from_numpy(x).cuda() for x in (a_id, a_val, b_id, b_val, b_g)]
    q3, t3 = timed(lambda: J.groupby_sum(d[0], d[1], d[2], d[4]))
    q4, t4 = timed(lambda: J.sum_product(d[0], d[1], d[2], d[3]))
    res["q3_groupby_sum_1Mx1M"] = {"seconds_per_call": t3, "rows_per_s": 2 * n / t3,
                                   "join_pairs": int(sum(c for _, _, c in q3)),
                                   "parity_exact": q3 == relational.groupby_sum(a_id, a_val,
                                                                                b_id, b_g)}
    res["q4_sum_product_1Mx1M"] = {"seconds_per_call": t4, "rows_per_s": 2 * n / t4,
                                   "join_pairs": q4[1],
                                   "parity_exact": q4 == relational.sum_product(a_id, a_val,
                                                                                b_id, b_val)}
    J.close()
    return res


def run_subs(args, data):
    """The other workloads, each a few steps, in the headline line."""
    import torch
    sub = {"note": "each workload a few steps; see its own bench workload for the full run"}
    sub["config1_2000x2000"] = guarded(run_config1, args)
    sub["fp8_threshold_join"] = guarded(run_fp8, args, data=data, steps=3, warmup=2)
    torch.cuda.empty_cache()
    sub["infonce_65536"] = guarded(run_infonce, args, steps=3, warmup=3, cpu_seconds=5.0)
    torch.cuda.empty_cache()
    sub["batch_4096_jobs"] = guarded(run_batch, args, steps=3, warmup=2, e2e=False)
    torch.cuda.empty_cache()
    sub["relational"] = guarded(run_relational, args)
    torch.cuda.empty_cache()
    sub["zipf_topk50_1Mx1M_fp8"] = guarded(run_zipf_child, args)
    return sub


def run_zipf_child(args):
    """The Zipf(1.1) top-50 join (d = 256, 50,000 centres) on 1M left rows
    against the full 1M right rows, E4M3 screen plus the precision cascade,
    as its own process (its own device memory); the per-row cost does not
    depend on the number of left rows (the cascade re-joins rows in chunks
    of 524,288).  500 cluster-stratified rows are checked against the
    oracle."""
    import subprocess
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "zipf", "--shape",
           "1000000,1000000", "--prec", "fp8", "--parity-rows", "500", "--steps", "2",
           "--warmup", "3", "--no-e2e"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("zipf run failed: " + r.stderr[-400:])
    line = [x for x in r.stdout.splitlines() if x.startswith("{")][-1]
    return json.loads(line)


def main():
    args = parse()
    if args.workload in ("infonce", "batch", "fp8", "relational") or \
            (args.workload == "zipf" and args.gpus > 1):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "workload": args.workload,
                              "unavailable": "the reference arm times the join workload"}))
            return 0
        if args.workload == "zipf":
            print(json.dumps({"workload": "zipf", "unavailable": "one-GPU workload"}))
            return 0
        fn = {"infonce": run_infonce, "batch": run_batch, "fp8": run_fp8,
              "relational": run_relational}[args.workload]
        print(json.dumps(fn(args)), flush=True)
        return 0
    if args.workload == "zipf":
        w = dict(ZIPF)
        if args.shape:
            nA, nB = (int(x) for x in args.shape.split(","))
            w.update(nA=nA, nB=nB, workload="topk_join_%dx%d_d256_k50_zipf1.1" % (nA, nB))
    else:
        w = dict(SMALL if args.small else WORKLOAD)
        if args.shape:
            nA, nB = (int(x) for x in args.shape.split(","))
            w.update(nA=nA, nB=nB, clusters=max(1, nB // 10),
                     workload="bf16_similarity_join_%dx%d_d768_k20_tau0.85" % (nA, nB))
    if args.prec:
        w["prec"] = args.prec
    if args.impl == "reference":
        return run_reference(args, w)

    import ctypes

    import torch

    from paper_2112_07552_gb300 import _build, sj

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _build.build()
    L = sj.lib()

    A, B, dups = make_data(w, rank)
    nA, nB, d, k = w["nA"], w["nB"], w["d"], w["k"]
    dev = torch.device("cuda", local)
    dA = torch.from_numpy(A).to(dev)
    dB = torch.from_numpy(B).to(dev)
    stream = torch.cuda.current_stream(dev)
    J = sj.SimilarityJoin(d, prec=w["prec"], device=local, stream=stream)
    thr = w["tau"] is not None
    cap = 40_000_000 if thr else 0
    idx = torch.empty((nA, k), dtype=torch.int64, device=dev)
    sc = torch.empty((nA, k), dtype=torch.float32, device=dev)
    pairs = torch.empty((max(cap, 1), 3), dtype=torch.int64, device=dev)
    n_out = sj.I64(0)

    def job(Ap, Bp, ip, sp, pp):
        jb = (sj.SjJob * 1)()
        jb[0].A, jb[0].nA, jb[0].B, jb[0].nB = Ap, nA, Bp, nB
        jb[0].k = k
        jb[0].topk_idx, jb[0].topk_score = ip, sp
        if thr:  # top-k only otherwise (no pair output)
            jb[0].tau = w["tau"]
            jb[0].pairs = pp
            jb[0].capacity = cap
            jb[0].n_out = ctypes.cast(ctypes.byref(n_out), sj.P)
        return jb

    jb_dev = job(dA.data_ptr(), dB.data_ptr(), idx.data_ptr(), sc.data_ptr(), pairs.data_ptr())

    def step(jb):
        st = sj.SjStats()
        code = L.sj_batch(J.handle, jb, 1, ctypes.byref(st))
        if code != sj.SJ_OK:
            raise sj.SJError(code, "sj_batch")
        return st

    for _ in range(args.warmup):
        step(jb_dev)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [step(jb_dev) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    value = world * nA * nB / (ms / 1e3)
    ms_score = statistics.mean(s.ms_score for s in stats)
    n_pairs = int(n_out.value)
    launches = int(sum(s.n_launches for s in stats))

    # end to end through the same call with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(A).pin_memory()
        hB = torch.from_numpy(B).pin_memory()
        hidx = torch.empty((nA, k), dtype=torch.int64).pin_memory()
        hsc = torch.empty((nA, k), dtype=torch.float32).pin_memory()
        hpairs = torch.empty((max(cap, 1), 3), dtype=torch.int64).pin_memory()
        jb_host = job(hA.data_ptr(), hB.data_ptr(), hidx.data_ptr(), hsc.data_ptr(),
                      hpairs.data_ptr())
        step(jb_host)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(jb_host)
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        if dist:
            t = torch.tensor([e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        e2e = {"value": world * nA * nB / (e_ms / 1e3), "unit": METRIC,
               "ms_per_step": e_ms,
               "h2d_bytes_per_step": int((nA + nB) * d * 4),
               "d2h_bytes_per_step": int(nA * k * 12 + int(n_out.value) * 24)}
        gpu_out = (hidx.numpy(), hsc.numpy(),
                   (hpairs[:n_pairs, 0].numpy(), hpairs[:n_pairs, 1].numpy(),
                    hpairs[:n_pairs, 2:3].view(torch.float32)[:, 0].numpy()))
    else:
        gpu_out = (idx.cpu().numpy(), sc.cpu().numpy(),
                   (pairs[:n_pairs, 0].cpu().numpy(), pairs[:n_pairs, 1].cpu().numpy(),
                    pairs[:n_pairs, 2:3].view(torch.float32)[:, 0].cpu().numpy()))

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    # tensor flops the scoring kernel issues: the hi/lo split multiplies 3d-wide rows
    flops = 2.0 * nA * nB * d * (3 if w["prec"] == "bf16x3" else 1)
    achieved = flops / (ms_score / 1e3) / 1e12
    bound, peak_source = "tensor", src + " bf16_tflops_sustained"
    if w["prec"] == "fp8":
        peak8 = guarded(fp8_peak_tflops)
        if isinstance(peak8, float):
            peak, peak_source = peak8, "measured here: torch._scaled_mm E4M3 8192^3, best of 5"
        else:
            peak, peak_source = 2.0 * peak, src + " bf16_tflops_sustained x 2 (nominal FP8/BF16)"
    elif w["prec"] == "fp32":
        # CUDA-core FMA rate: SMs x 128 FP32 lanes x 2 flop x the SM clock seen
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        bound, peak = "alu", sms * 128 * 2 * mhz * 1e6 / 1e12
        peak_source = "derived: %d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (sampled)" % (sms, mhz)
    cpu = None
    if world == 1 and not args.no_cpu and args.workload != "zipf":
        cpu = cpu_baseline(w, A, B, args.cpu_seconds, gpu_out, dups)
    fp8_sample = zipf_par = None
    if args.workload == "zipf" and world == 1:
        fp8_sample = guarded(fp8_error_sample, w, A, B, dB)
        if not args.no_cpu:
            zipf_par = guarded(zipf_parity, w, A, B, gpu_out[0], gpu_out[1], args.parity_rows)
    headline = args.workload == "join" and not args.shape and not args.small
    # algorithmic bytes of one scoring launch: the packed operands read once
    # plus the band lists written once (the k best of each list and its
    # margin band); the measured DRAM traffic is compared against it
    elem = {"fp8": 1, "fp32": 4, "bf16x3": 6}.get(w["prec"], 2)
    algo_bytes = float((nA + nB) * d * elem + nA * 2 * (2 * k + 64) * 8)
    traffic, traffic_src = (score_tc_traffic(float(nA) * nB) if w["prec"] == "bf16"
                            else (None, "not captured for this precision"))
    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp8": "e4m3"}.get(w["prec"], w["prec"]), "data": "synthetic",
        "config": join_config(w, world),
        "roofline": {"bound": bound,
                     "kernel": "score_simt_kernel" if w["prec"] == "fp32" else "score_tc_kernel",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "peak_source": peak_source,
                     "traffic": traffic, "traffic_source": traffic_src,
                     "traffic_per_algorithmic_byte": (traffic / algo_bytes) if traffic else None,
                     "algorithmic_bytes": algo_bytes, "ms_kernel": ms_score},
        "stages_ms": {"prepare": statistics.mean(s.ms_prepare for s in stats),
                      "score": ms_score,
                      "select": statistics.mean(s.ms_select for s in stats)},
        "n_pairs": n_pairs,
        "n_candidates": int(stats[-1].n_candidates),
        "n_exact": int(stats[-1].n_exact),
        "n_rescored": int(stats[-1].n_rescored),
        "n_tier2_rows": int(stats[-1].n_tier2_rows),
        "n_overflow_rows": int(stats[-1].n_overflow_rows),
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        # largest observed |s~ - s| over rescored candidates and largest proven
        # margin, in the scoring precision of this line
        "max_abs_err_lowprec": float(stats[-1].max_abs_err_lowprec),
        "margin_max": float(stats[-1].margin_max),
    }
    if fp8_sample is not None:
        out["fp8_error_vs_fp64"] = fp8_sample
    if zipf_par is not None:
        out["parity_stratified"] = zipf_par
        if "oracle_pair_scores_per_s" in zipf_par:
            out["cpu_baseline"] = {"value": zipf_par["oracle_pair_scores_per_s"], "unit": METRIC,
                                   "cores": zipf_par["oracle_cores"], "kind": "oracle",
                                   "sample": "%d cluster-stratified left rows x all %d right rows "
                                             "(top-%d), %.1f s" % (zipf_par["rows"], nB, k,
                                                                   zipf_par["oracle_seconds"]),
                                   "parity_rows_exact": zipf_par["exact"]}
    if args.workload == "zipf":
        nxt = "the BF16 hi/lo split with band lists sized by their columns"
        out["fallback_share"] = {
            "rows": int(stats[-1].n_overflow_rows),
            "fraction": stats[-1].n_overflow_rows / nA,
            "how": "rows whose band lists overflowed on the first pass, re-joined in " + nxt,
            "rejoined_rows": int(stats[-1].n_rejoined_rows),
            "rejoined_again": int(stats[-1].n_rejoined_again),
            "rejoined_again_how": "lists overflowed there too: re-joined in FP32"}
    if headline and world == 1 and not args.no_sub:
        out["fp32_same_join"] = guarded(fp32_same_join, args, w, dA, dB, stream, idx, sc,
                                        gpu_out[2], value)
        out["planner"] = guarded(lambda: dict(J.plan(dA, dB, k, w["tau"]),
                                              measured_ms_bf16=ms))
        J.close()
        del idx, sc, pairs
        torch.cuda.empty_cache()
        out["sub"] = run_subs(args, (A, B, dA, dB))
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
