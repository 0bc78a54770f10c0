"""The precision planner (sj_plan): its choice is (close to) the fastest
precision measured on the full join, and every precision emits the same
results.  Three workloads where the answer differs: a clustered top-k +
threshold join (BF16: E4M3's margin overflows the top-k lists), a threshold
join alone (E4M3: its margin stays selective above tau and it issues twice
the BF16 rate) and a top-50 join inside one dense cluster (the BF16 hi/lo
split: the BF16 margin band overflows the lists into rescans of all of B)."""
import time

import numpy as np
import pytest

from paper_2112_07552_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sjmod():
    from paper_2112_07552_gb300 import _build, sj
    _build.build()
    return sj


def clustered(nA, nB, d, K, seed, near_dup=True):
    C = datagen.centres(K, d, seed)
    A = datagen.clustered(nA, d, K, 0.1, seed, stream=0, C=C)
    B = datagen.clustered(nB, d, K, 0.1, seed, stream=1, C=C)
    if near_dup:
        datagen.add_near_duplicates(A, B, 0.05, 0.02, seed)
    return A, B


def measure(sjmod, A, B, k, tau, prec, reps=2):
    d = A.shape[1]
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    job = {"A": dA, "B": dB}
    if k:
        job["k"] = k
    if tau is not None:
        job["tau"] = tau
        job["capacity"] = 64 * A.shape[0]
    with sjmod.SimilarityJoin(d, prec=prec, device=0) as J:
        out = J.batch([job])  # warm-up (workspace)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            out = J.batch([job])
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / reps
    return ms, {key: v.cpu().numpy() for key, v in out[0].items()}


@pytest.mark.parametrize("case", ["topk_and_threshold", "threshold_only", "dense_top50"])
def test_plan_choice_is_near_fastest_and_results_agree(sjmod, case):
    if case == "dense_top50":
        A, B = clustered(4096, 120_000, 256, 1, 80, near_dup=False)
        k, tau = 50, None
    else:
        A, B = clustered(16384, 200_000, 768, 20_000, 81)
        k, tau = (20, 0.85) if case == "topk_and_threshold" else (0, 0.85)
    with sjmod.SimilarityJoin(A.shape[1], prec="bf16", device=0) as J:
        plan = J.plan(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), k, tau)
    times, outs = {}, {}
    for prec in ("bf16", "fp8", "bf16x3", "fp32"):
        times[prec], outs[prec] = measure(sjmod, A, B, k, tau, prec)
    print(case, plan["choice"], {p: round(v, 1) for p, v in plan["est_ms"].items()},
          {p: round(v, 1) for p, v in times.items()})
    best = min(times.values())
    assert times[plan["choice"]] <= 1.25 * best, (plan, times)
    for prec in ("fp8", "bf16x3", "fp32"):
        for key in outs["bf16"]:
            assert np.array_equal(outs[prec][key], outs["bf16"][key]), (prec, key)
