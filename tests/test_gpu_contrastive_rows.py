"""The row-sharded contrastive join (sj_contrastive_fwd_rows /
sj_backward_rows) on one GPU: the ranks of a data-parallel run are emulated
one after the other (their calls do not wait on each other), their loss parts
and dB contributions summed as the all-reduce would, and everything compared
with the FP64 oracle of the whole join (tolerances as in
test_gpu_contrastive.py)."""
import numpy as np
import pytest

import oracle
from paper_2112_07552_gb300 import datagen, shard
from test_gpu_contrastive import bf16_inputs, check_grad, grad_bounds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sjmod():
    from paper_2112_07552_gb300 import _build, sj
    _build.build()
    return sj


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("N,d,T,world", [(1000, 96, 0.05, 3), (640, 448, 0.1, 2),
                                         (4096, 768, 0.05, 4)])
def test_row_shards_sum_to_the_whole_join(sjmod, N, d, T, world, fused):
    A, B = datagen.paired(N, d, max(2, N // 8), seed=N + d + world)
    ab, bb = bf16_inputs(A, B)
    loss_w, lse_w, _, dA_w, dB_w = oracle.infonce(ab, bb, T, g=1.0)
    flags = sjmod.SJ_FLAG_FUSED_BACKWARD if fused else 0
    dBt = torch.from_numpy(B).cuda()
    loss, lse, dA, dB = 0.0, [], [], None
    with sjmod.SimilarityJoin(d, prec="bf16", device=0, flags=flags) as J:
        fwd, bwd = shard.library_rows(J)
        for rank in range(world):
            r0, r1 = shard.row_range(N, rank, world)
            lp, l, ga, gb = shard.infonce_step(fwd, bwd, torch.from_numpy(A[r0:r1]).cuda(), r0,
                                               dBt, T)
            loss += float(lp.item())
            lse.append(l.cpu().numpy())
            dA.append(ga.cpu().numpy())
            gb = gb.cpu().numpy().astype(np.float64)
            dB = gb if dB is None else dB + gb  # the all-reduce of dB
    lse = np.concatenate(lse)
    assert abs(loss - loss_w) <= 5e-5 * max(1.0, abs(loss_w))
    assert np.max(np.abs(lse - lse_w)) <= 5e-5 * max(1.0, np.max(np.abs(lse_w)))
    bA, bB = grad_bounds(ab, bb, T, False, 1.0, np.abs(lse - lse_w))
    check_grad(np.concatenate(dA), dA_w, bA)
    check_grad(dB, dB_w, bB + world * 2.0 ** -23 * np.abs(dB_w))  # + the parts' float sum


def test_row_shard_arguments(sjmod):
    A, B = datagen.paired(64, 32, 8, seed=3)
    with sjmod.SimilarityJoin(32, prec="bf16", device=0) as J:
        with pytest.raises(sjmod.SJError) as e:  # r0 + n_rows > N
            J.contrastive_forward_rows(torch.from_numpy(A[:40]).cuda(), 30,
                                       torch.from_numpy(B).cuda(), 0.1)
        assert e.value.code == sjmod.SJ_ERR_INVALID_ARG
    with sjmod.SimilarityJoin(32, prec="bf16", device=0, flags=sjmod.SJ_FLAG_SYM_INFONCE) as J:
        with pytest.raises(sjmod.SJError) as e:
            J.contrastive_forward_rows(torch.from_numpy(A[:8]).cuda(), 0,
                                       torch.from_numpy(B).cuda(), 0.1)
        assert e.value.code == sjmod.SJ_ERR_UNSUPPORTED
