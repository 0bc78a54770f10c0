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

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _data(seed, nA, nB, d):
    from paper_2112_07552_gb300 import datagen
    A = datagen.clustered(nA, d, 20, 0.1, seed=seed, stream=0)
    B = datagen.clustered(nB, d, 20, 0.1, seed=seed, stream=1)
    return torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()


def test_noalloc_matches_sj_topk_on_two_calls_in_a_row():
    from paper_2112_07552_gb300 import _build, sj
    _build.build()
    L = sj.lib()
    stream = torch.cuda.current_stream().cuda_stream
    # two different joins back to back: the second must not see the first's
    # scratch contents
    for seed, nA, nB, d, k in ((31, 300, 1500, 64, 12), (32, 129, 2048, 96, 5)):
        dA, dB = _data(seed, nA, nB, d)
        with sj.SimilarityJoin(d, prec="bf16", device=0) as J:
            ref_idx, ref_sc = J.topk(dA, dB, k)
        idx = torch.full((nA, k), -7, dtype=torch.int64, device="cuda")
        sc = torch.full((nA, k), 7.0, dtype=torch.float32, device="cuda")
        code = L.sj_topk_noalloc(dA.data_ptr(), nA, dB.data_ptr(), nB, d, k, idx.data_ptr(),
                                 sc.data_ptr(), stream)
        assert code == sj.SJ_OK, sj.status_string(code)
        # the same tolerance as every parity test here: bit-exact
        assert torch.equal(idx, ref_idx)
        assert np.array_equal(sc.cpu().numpy().view(np.uint32),
                              ref_sc.cpu().numpy().view(np.uint32))


def test_noalloc_rejects_sizes_over_its_limit():
    from paper_2112_07552_gb300 import sj
    L = sj.lib()
    dA, _ = _data(33, 10, 10, 16)
    big = torch.zeros((2049, 16), dtype=torch.float32, device="cuda")
    idx = torch.empty((10, 3), dtype=torch.int64, device="cuda")
    sc = torch.empty((10, 3), dtype=torch.float32, device="cuda")
    code = L.sj_topk_noalloc(dA.data_ptr(), 10, big.data_ptr(), 2049, 16, 3, idx.data_ptr(),
                             sc.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert code == sj.SJ_ERR_UNSUPPORTED
