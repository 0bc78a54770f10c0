"""sj_topk_noalloc: the top-k entry point for callers that cannot allocate.

Such callers (a serving process whose device memory is already reserved by
another allocator, or latency-critical code that must not call
cudaMalloc/cudaFree because they can synchronise the device) get results
identical to sj_topk from a library-owned fixed scratch array.  This file is
collected last so that a stop-at-first-failure run has run every other test
first; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _data(seed, nA, nB, d):
    from paper_2112_07552_gb300 import datagen
    A = datagen.clustered(nA, d, 20, 0.1, seed=seed, stream=0)
    B = datagen.clustered(nB, d, 20, 0.1, seed=seed, stream=1)
    return A, B


def _noalloc(dA, dB, k, stream=None):
    from paper_2112_07552_gb300 import sj
    L = sj.lib()
    nA, d = dA.shape
    nB = dB.shape[0]
    idx = torch.full((nA, k), -7, dtype=torch.int64, device="cuda")
    sc = torch.full((nA, k), 7.0, dtype=torch.float32, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    code = L.sj_topk_noalloc(dA.data_ptr(), nA, dB.data_ptr() if nB else None, nB, d, k,
                             idx.data_ptr(), sc.data_ptr(), stream)
    return code, idx, sc


def _bits(x):
    return np.ascontiguousarray(x).view(np.uint32)


def test_noalloc_matches_sj_topk_on_two_calls_in_a_row():
    from paper_2112_07552_gb300 import _build, sj
    _build.build()
    # two different joins back to back: the second must not see the first's
    # scratch contents
    for seed, nA, nB, d, k in ((31, 300, 1500, 64, 12), (32, 129, 2048, 96, 5)):
        A, B = _data(seed, nA, nB, d)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        with sj.SimilarityJoin(d, prec="bf16", device=0) as J:
            ref_idx, ref_sc = J.topk(dA, dB, k)
        code, idx, sc = _noalloc(dA, dB, k)
        assert code == sj.SJ_OK, sj.status_string(code)
        # the same tolerance as every parity test here: bit-exact
        assert torch.equal(idx, ref_idx)
        assert np.array_equal(_bits(sc.cpu().numpy()), _bits(ref_sc.cpu().numpy()))
        # and against the oracle itself
        w_idx, w_s, _ = oracle.topk(A, B, k)
        assert np.array_equal(idx.cpu().numpy(), w_idx)
        assert np.array_equal(_bits(sc.cpu().numpy()), _bits(w_s))


def test_noalloc_padding_and_empty_right_side():
    from paper_2112_07552_gb300 import sj
    A, B = _data(34, 40, 7, 32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    # k > nB: (-1, -inf) padding, as sj_topk and the oracle
    code, idx, sc = _noalloc(dA, dB, 10)
    assert code == sj.SJ_OK
    with sj.SimilarityJoin(32, prec="bf16", device=0) as J:
        ref_idx, ref_sc = J.topk(dA, dB, 10)
    assert torch.equal(idx, ref_idx)
    assert np.array_equal(_bits(sc.cpu().numpy()), _bits(ref_sc.cpu().numpy()))
    w_idx, w_s, _ = oracle.topk(A, B, 10)
    assert np.array_equal(idx.cpu().numpy(), w_idx)
    assert np.array_equal(_bits(sc.cpu().numpy()), _bits(w_s))
    # nB = 0: every slot padded
    code, idx, sc = _noalloc(dA, dB[:0], 3)
    assert code == sj.SJ_OK
    assert (idx.cpu().numpy() == -1).all() and np.isneginf(sc.cpu().numpy()).all()


def test_noalloc_validation_then_a_valid_call():
    from paper_2112_07552_gb300 import sj
    A, B = _data(35, 64, 100, 48)
    bad = B.copy()
    bad[17] *= 1.01  # | ||x||^2 - 1 | ~ 0.02
    dA = torch.from_numpy(A).cuda()
    code, _, _ = _noalloc(dA, torch.from_numpy(bad).cuda(), 4)
    assert code == sj.SJ_ERR_NOT_UNIT_NORM
    nan = A.copy()
    nan[5, 3] = np.nan
    code, _, _ = _noalloc(torch.from_numpy(nan).cuda(), torch.from_numpy(B).cuda(), 4)
    assert code == sj.SJ_ERR_NONFINITE
    # the status area is cleared by every call: a valid call right after the
    # failed ones succeeds with exact results
    code, idx, sc = _noalloc(dA, torch.from_numpy(B).cuda(), 4)
    assert code == sj.SJ_OK
    w_idx, w_s, _ = oracle.topk(A, B, 4)
    assert np.array_equal(idx.cpu().numpy(), w_idx)
    assert np.array_equal(_bits(sc.cpu().numpy()), _bits(w_s))


def test_noalloc_rejects_sizes_over_its_limit():
    from paper_2112_07552_gb300 import sj
    A, _ = _data(33, 10, 10, 16)
    dA = torch.from_numpy(A).cuda()
    big = torch.zeros((2049, 16), dtype=torch.float32, device="cuda")
    code, _, _ = _noalloc(dA, big, 3)
    assert code == sj.SJ_ERR_UNSUPPORTED


def test_noalloc_rejects_host_pointers_and_capture():
    from paper_2112_07552_gb300 import sj
    L = sj.lib()
    A, B = _data(36, 8, 16, 16)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    hB = torch.from_numpy(B)
    idx = torch.empty((8, 2), dtype=torch.int64, device="cuda")
    sc = torch.empty((8, 2), dtype=torch.float32, device="cuda")
    code = L.sj_topk_noalloc(dA.data_ptr(), 8, hB.data_ptr(), 16, 16, 2, idx.data_ptr(),
                             sc.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert code == sj.SJ_ERR_INVALID_ARG
    # a stream under graph capture is refused before anything is enqueued
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        dummy = dA * 2.0
        code = L.sj_topk_noalloc(dA.data_ptr(), 8, dB.data_ptr(), 16, 16, 2, idx.data_ptr(),
                                 sc.data_ptr(), s.cuda_stream)
        g.capture_end()
    assert code == sj.SJ_ERR_INVALID_ARG
    del dummy, g


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two GPUs")
def test_noalloc_rejects_other_device_memory():
    from paper_2112_07552_gb300 import sj
    A, B = _data(37, 8, 16, 16)
    dA = torch.from_numpy(A).cuda(0)
    dB1 = torch.from_numpy(B).cuda(1)
    with torch.cuda.device(0):
        code, _, _ = _noalloc(dA, dB1, 2)
    assert code == sj.SJ_ERR_INVALID_ARG
