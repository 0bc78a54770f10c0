"""Block-sparse scoring (SJ_FLAG_BLOCK_SPARSE; the paper's answer to low
density, Sec. 4.3): the same joins with and without the flag emit identical
results, equal to the oracle's, on dense rows, on high-cardinality one-hot
keys in key order (most tiles share no nonzero k-block) and in random order,
and on rows whose nonzeros fall in few k-blocks; the sorted one-hot threshold
join is faster with the flag."""
import time

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


def run(sjmod, A, B, k, tau, flags, prec="bf16", reps=1):
    d = A.shape[1]
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    job = {"A": dA, "B": dB}
    if k:
        job["k"] = k
    if tau is not None:
        job["tau"] = tau
        job["capacity"] = max(1024, 64 * A.shape[0])
    with sjmod.SimilarityJoin(d, prec=prec, device=0, flags=flags) as J:
        out, st = J.batch([job], with_stats=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            out = J.batch([job])
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / reps
    return {key: v.cpu().numpy() for key, v in out[0].items()}, ms


def same(a, b):
    return all(np.array_equal(a[key], b[key]) for key in a)


def one_hot_rows(n, n_keys, seed, stream, order):
    keys = datagen.keys(n, n_keys, seed, stream)
    if order == "sorted":
        keys = np.sort(keys)
    return keys, datagen.one_hot(keys, n_keys)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("order", ["sorted", "random"])
def test_one_hot_high_cardinality(sjmod, prec, order):
    ka, A = one_hot_rows(1500, 3000, 1, 0, order)
    kb, B = one_hot_rows(2500, 3000, 1, 1, order)
    for k, tau in ((0, 0.5), (3, None), (2, 0.5)):
        dense, _ = run(sjmod, A, B, k, tau, 0, prec)
        sparse, _ = run(sjmod, A, B, k, tau, sjmod.SJ_FLAG_BLOCK_SPARSE, prec)
        assert same(dense, sparse), (k, tau)
        if tau is not None:
            wi, wj, ws, _ = oracle.threshold(A, B, tau, want_s64=False)
            assert np.array_equal(sparse["i"], wi) and np.array_equal(sparse["j"], wj)
            assert np.array_equal(sparse["pair_score"].view(np.uint32), ws.view(np.uint32))
        if k:
            wi, ws, _ = oracle.topk(A, B, k)
            assert np.array_equal(sparse["idx"], wi)
            assert np.array_equal(sparse["score"].view(np.uint32), ws.view(np.uint32))


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
def test_dense_and_few_block_rows_unchanged(sjmod, prec):
    A = datagen.clustered(700, 320, 30, 0.1, seed=5, stream=0)
    B = datagen.clustered(900, 320, 30, 0.1, seed=5, stream=1)
    # rows whose nonzeros lie in one 64-wide block (zero elsewhere)
    C = np.zeros((300, 320), np.float32)
    for t in range(300):
        blk = t % 5
        v = np.random.default_rng(t).standard_normal(64)
        C[t, blk * 64:(blk + 1) * 64] = v / np.linalg.norm(v)
    for X, Y in ((A, B), (C, B), (A, C), (C, C)):
        dense, _ = run(sjmod, X, Y, 5, 0.3, 0, prec)
        sparse, _ = run(sjmod, X, Y, 5, 0.3, sjmod.SJ_FLAG_BLOCK_SPARSE, prec)
        assert same(dense, sparse)
        wi, ws, _ = oracle.topk(X, Y, 5)
        assert np.array_equal(sparse["idx"], wi)


def test_sorted_one_hot_threshold_is_faster(sjmod):
    # 8,192 x 32,768 rows over 32,768 keys in key order: the dense tiles
    # multiply d = 32,768 one-hot columns; nearly all of them are zero
    ka, A = one_hot_rows(8192, 32768, 2, 0, "sorted")
    kb, B = one_hot_rows(32768, 32768, 2, 1, "sorted")
    dense, t_dense = run(sjmod, A, B, 0, 0.5, 0, reps=2)
    sparse, t_sparse = run(sjmod, A, B, 0, 0.5, sjmod.SJ_FLAG_BLOCK_SPARSE, reps=2)
    assert same(dense, sparse)
    print("dense %.1f ms, block-sparse %.1f ms" % (t_dense, t_sparse))
    assert t_sparse < 0.5 * t_dense
