"""Parity at the sizes where the kernels take paths small joins never reach.

* A multi-wave join from the headline generator: 131,035 x 1,000,000,
  d = 768, 100,000 centres, 5% near duplicates, k = 20 and tau = 0.85 in one
  fused call.  Each CTA scores several row blocks (the accumulator phase
  carries across units), every row's lists cover 500,000 columns, and the
  last row block is ragged.  The sample is 128 rows that have a near
  duplicate in B, 128 random rows and the last 16 rows, compared bit for bit
  with the oracle.
* A short left side against the same 1,000,000 rows (2,000 x 1,000,000): the
  planner splits every row block's columns about 20 ways, so each row's
  candidates come from about 40 lists.
* The contrastive join at N = 16,384, d = 768: loss, every lse and every
  entry of dA and dB against the FP64 oracle (tolerances as in
  test_gpu_contrastive.py), for both backward paths.
"""
import numpy as np
import pytest

import oracle
from paper_2112_07552_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sjmod():
    from paper_2112_07552_gb300 import _build, sj
    _build.build()
    return sj


@pytest.fixture(scope="module")
def headline_data():
    nA, nB, d, K = 131_035, 1_000_000, 768, 100_000
    C = datagen.centres(K, d, 0)
    A = datagen.clustered(nA, d, K, 0.1, 0, stream=0, C=C)
    B = datagen.clustered(nB, d, K, 0.1, 0, stream=1, C=C)
    dups = datagen.add_near_duplicates(A, B, 0.05, 0.02, 0)
    return A, B, dups


def fused_join(sjmod, A, B, k, tau):
    d = A.shape[1]
    with sjmod.SimilarityJoin(d, prec="bf16", device=0) as J:
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        # room for 40 pairs per row: one call, no capacity retry
        out, st = J.batch([{"A": dA, "B": dB, "k": k, "tau": tau, "capacity": 40 * A.shape[0]}],
                          with_stats=True)
        o = {key: v.cpu().numpy() for key, v in out[0].items()}
    torch.cuda.synchronize()
    return o, st


def check_rows(o, A, B, k, tau, rows):
    idx, s32, _ = oracle.topk(A, B, k, rows=rows)
    gi, gs = o["idx"][rows], o["score"][rows]
    bad = np.nonzero((gi != idx).any(axis=1) |
                     (gs.view(np.uint32) != s32.view(np.uint32)).any(axis=1))[0]
    assert bad.size == 0, "top-k rows %s differ" % rows[bad[:5]]
    ti, tj, ts, _ = oracle.threshold(A, B, tau, rows=rows, want_s64=False)
    sel = np.isin(o["i"], rows)
    assert np.array_equal(o["i"][sel], ti) and np.array_equal(o["j"][sel], tj)
    assert np.array_equal(o["pair_score"][sel].view(np.uint32), ts.view(np.uint32))


def test_join_131035x1M_multiwave_sampled_rows(sjmod, headline_data):
    A, B, dups = headline_data
    k, tau = 20, 0.85
    o, st = fused_join(sjmod, A, B, k, tau)
    nA = A.shape[0]
    rng = np.random.default_rng(2024)
    with_dup = np.unique(dups[:, 0][dups[:, 0] < nA])
    rows = np.unique(np.concatenate([
        rng.choice(with_dup, size=128, replace=False),
        rng.choice(nA, size=128, replace=False),
        np.arange(nA - 16, nA)]))
    check_rows(o, A, B, k, tau, rows)
    # every sampled near-duplicate row finds its partner first (cosine ~0.9998)
    part = dict(map(tuple, dups))
    for i in rows:
        if i in part:
            assert o["idx"][i, 0] == part[i]
    assert st["n_overflow_rows"] == 0 and st["n_pairs"] == len(o["i"])


def test_join_2000x1M_many_column_splits(sjmod, headline_data):
    A, B, dups = headline_data
    A2 = np.ascontiguousarray(A[:2000])
    k, tau = 20, 0.85
    o, st = fused_join(sjmod, A2, B, k, tau)
    rng = np.random.default_rng(2025)
    with_dup = np.unique(dups[:, 0][dups[:, 0] < 2000])
    rows = np.unique(np.concatenate([rng.choice(with_dup, size=min(24, len(with_dup)),
                                                replace=False),
                                     rng.choice(2000, size=40, replace=False), [1999]]))
    check_rows(o, A2, B, k, tau, rows)
    assert st["n_candidates"] > 0


@pytest.fixture(scope="module")
def case_16384():
    from test_gpu_contrastive import bf16_inputs
    N, d, T = 16384, 768, 0.05
    A, B = datagen.paired(N, d, 2000, seed=46)
    ab, bb = bf16_inputs(A, B)
    return A, B, ab, bb, T, oracle.infonce(ab, bb, T, g=1.0)


@pytest.mark.parametrize("fused", [False, True])
def test_contrastive_16384_full(sjmod, case_16384, fused):
    from test_gpu_contrastive import check_grad, grad_bounds, run
    A, B, ab, bb, T, want = case_16384
    loss_w, lse_w, _, dA_w, dB_w = want
    loss, lse, gA, gB = run(sjmod, A, B, T, fused=fused)
    assert abs(loss - loss_w) <= 5e-5 * max(1.0, abs(loss_w))
    assert np.max(np.abs(lse - lse_w)) <= 5e-5 * max(1.0, np.max(np.abs(lse_w)))
    bA, bB = grad_bounds(ab, bb, T, False, 1.0, np.abs(lse - lse_w))
    check_grad(gA, dA_w, bA)
    check_grad(gB, dB_w, bB)
