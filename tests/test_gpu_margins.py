"""The error-bound invariant on every pair: |s~_ij - s_ij| <= m_i.

The exactness of every emitted result rests on the margin m_i the fused
filter uses (the band below the running k-th score and the threshold
candidates are both m_i wide).  Its accumulation term is an allowance for the
tensor core's undocumented FP32 (BF16) and FP8 accumulation.  These tests
read back the raw low-precision score of EVERY pair of small joins
(sj_debug_scores) and check it against the oracle's FP64 enclosure of the
exact score: s~ - lo <= m and hi - s~ <= m, for BF16, E4M3, the BF16 hi/lo
split and the FP32 CUDA-core form, on clustered data and on rows built to
stress accumulation (long same-sign runs cancelled by one large term, half
the coordinates cancelling the other half, exponents spread over 2^-20..2^0,
alternating signs).
"""
import numpy as np
import pytest

import oracle
from paper_2112_07552_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["bf16", "fp8", "bf16x3", "fp32"]


def raw_scores(prec, A, B, k=4):
    from paper_2112_07552_gb300 import sj
    L = sj.lib()
    nA, nB, d = A.shape[0], B.shape[0], A.shape[1]
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    raw = torch.full((nA, nB), float("nan"), dtype=torch.float32, device="cuda")
    marg = torch.full((nA,), float("nan"), dtype=torch.float32, device="cuda")
    with sj.SimilarityJoin(d, prec=prec, device=0) as J:
        code = L.sj_debug_scores(J.handle, raw.data_ptr(), marg.data_ptr())
        assert code == sj.SJ_OK, sj.status_string(code)
        idx, sc = J.topk(dA, dB, k)
    torch.cuda.synchronize()
    # the armed call still returns the exact top-k
    w_idx, w_s, _ = oracle.topk(A, B, k)
    assert np.array_equal(idx.cpu().numpy(), w_idx)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), w_s.view(np.uint32))
    return raw.cpu().numpy().astype(np.float64), marg.cpu().numpy().astype(np.float64)


def check_every_pair(prec, A, B):
    raw, m = raw_scores(prec, A, B)
    assert np.isfinite(raw).all(), "a pair's raw score was not written"
    assert np.isfinite(m).all() and (m > 0).all()
    lo, hi = oracle.enclose_all(A, B)
    err = np.maximum(raw - lo, hi - raw)  # >= |s~ - s| for the exact s in [lo, hi]
    ratio = err / m[:, None]
    worst = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert ratio.max() <= 1.0, (
        "%s: pair %s has |s~ - s| = %.3g > m_i = %.3g" % (prec, worst, err[worst], m[worst[0]]))
    return float(ratio.max()), float(np.abs(raw - 0.5 * (lo + hi)).max()), float(m.max())


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,d", [(2048, 256), (1024, 768)])
def test_margin_holds_on_every_pair_clustered(prec, n, d):
    A = datagen.clustered(n, d, max(1, n // 10), 0.1, seed=n + d, stream=0)
    B = datagen.clustered(n + 77, d, max(1, n // 10), 0.1, seed=n + d, stream=1)
    datagen.add_near_duplicates(A, B, 0.05, 0.02, seed=n + d)
    r, e, m = check_every_pair(prec, A, B)
    print("clustered %s n=%d d=%d: max err/m %.3g, max |s~-s| %.3g, max m %.3g"
          % (prec, n, d, r, e, m))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", datagen.ADVERSARIAL_KINDS)
@pytest.mark.parametrize("d", [256, 768])
def test_margin_holds_on_every_pair_adversarial(prec, kind, d):
    A = datagen.adversarial(640, d, kind, seed=d, side=0)
    B = datagen.adversarial(700, d, kind, seed=d, side=1)
    r, e, m = check_every_pair(prec, A, B)
    print("%s %s d=%d: max err/m %.3g, max |s~-s| %.3g, max m %.3g" % (kind, prec, d, r, e, m))
