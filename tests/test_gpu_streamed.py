"""Joins against a right table in host memory, streamed through the device
in row chunks (sj_topk_streamed, sj_threshold_streamed): identical to the
in-memory joins and to the oracle, including ties across chunks (exact
duplicate rows of B in different chunks: equal scores, lower index first;
rows differing by one ulp: equal float32 scores, different exact values),
with B pinned by the caller or pageable, and ragged last chunks."""
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


@pytest.fixture(scope="module")
def data():
    nA, nB, d = 600, 90_000, 128
    A = datagen.clustered(nA, d, 60, 0.1, seed=21, stream=0)
    B = datagen.clustered(nB, d, 60, 0.1, seed=21, stream=1)
    # copies of A's rows' best partners spread over chunks: exact duplicates
    # and one-ulp neighbours of some rows, far apart in B
    rng = np.random.default_rng(5)
    src = rng.choice(nB, size=400, replace=False)
    for t, s in enumerate(src):
        dst = (s + 37_000 * (1 + t % 2)) % nB
        B[dst] = B[s]
        if t % 3 == 0:
            k = int(rng.integers(d))
            B[dst, k] = np.nextafter(B[dst, k], np.float32(2.0))
    return A, B


@pytest.mark.parametrize("k,chunk", [(10, 40_000), (64, 25_000), (5, 90_000)])
def test_topk_streamed_equals_in_memory_and_oracle(sjmod, data, k, chunk):
    A, B = data
    dA = torch.from_numpy(A).cuda()
    with sjmod.SimilarityJoin(A.shape[1], prec="bf16", device=0) as J:
        ref_i, ref_s = J.topk(dA, torch.from_numpy(B).cuda(), k)
        for Bh in (B, torch.from_numpy(B).pin_memory()):  # pageable, pinned
            i, s = J.topk_streamed(dA, Bh, k, chunk_rows=chunk)
            assert torch.equal(i, ref_i)
            assert torch.equal(s.view(torch.int32), ref_s.view(torch.int32))
    rows = np.arange(0, A.shape[0], 7)
    wi, ws, _ = oracle.topk(A, B, k, rows=rows)
    assert np.array_equal(i.cpu().numpy()[rows], wi)
    assert np.array_equal(s.cpu().numpy()[rows].view(np.uint32), ws.view(np.uint32))


def test_threshold_streamed_equals_in_memory_and_oracle(sjmod, data):
    A, B = data
    with sjmod.SimilarityJoin(A.shape[1], prec="bf16", device=0) as J:
        ri, rj, rs = J.threshold(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 0.8)
        i, j, s = J.threshold_streamed(A, B, 0.8, chunk_rows=33_333)
    assert np.array_equal(i.numpy(), ri.cpu().numpy()) and np.array_equal(j.numpy(), rj.cpu().numpy())
    assert np.array_equal(s.numpy().view(np.uint32), rs.cpu().numpy().view(np.uint32))
    wi, wj, ws, _ = oracle.threshold(A, B, 0.8, want_s64=False)
    assert np.array_equal(i.numpy(), wi) and np.array_equal(j.numpy(), wj)


def test_streamed_refuses_device_B(sjmod, data):
    A, B = data
    with sjmod.SimilarityJoin(A.shape[1], prec="bf16", device=0) as J:
        with pytest.raises(sjmod.SJError) as e:
            J.topk_streamed(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 5)
        assert e.value.code == sjmod.SJ_ERR_INVALID_ARG


def test_streamed_overlaps_copies(sjmod):
    # 16,384 x 2,000,000 rows, d = 768 (B: 6.1 GB in pinned host memory) in
    # chunks of 262,144 rows, against the same join with B resident
    A = datagen.clustered(16384, 768, 2000, 0.1, seed=22, stream=0)
    B = torch.from_numpy(datagen.clustered(2_000_000, 768, 200_000, 0.1, seed=22,
                                           stream=1)).pin_memory()
    dA = torch.from_numpy(A).cuda()
    with sjmod.SimilarityJoin(768, prec="bf16", device=0) as J:
        J.topk_streamed(dA, B, 20, chunk_rows=262_144)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        i, s = J.topk_streamed(dA, B, 20, chunk_rows=262_144)
        torch.cuda.synchronize()
        t_stream = time.perf_counter() - t0
        dB = B.cuda()
        ri, rs = J.topk(dA, dB, 20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ri, rs = J.topk(dA, dB, 20)
        torch.cuda.synchronize()
        t_mem = time.perf_counter() - t0
    assert torch.equal(i, ri) and torch.equal(s.view(torch.int32), rs.view(torch.int32))
    print("streamed %.1f ms, resident %.1f ms (B 6.1 GB over the host link)"
          % (t_stream * 1e3, t_mem * 1e3))
