"""Multi-rank host logic with gloo ranks on CPU (world size 2).

Each rank joins its row shard of A against all of B with the oracle; the
gathered results must equal the unsharded join.  The contrastive reductions
(loss all-reduce, column logsumexp combine) are checked against the oracle's
unsharded values.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_2112_07552_gb300 import datagen, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = datagen.clustered(301, 32, 12, 0.1, seed=51, stream=0)
    B = datagen.clustered(257, 32, 12, 0.1, seed=51, stream=1)
    r0, r1 = shard.row_range(A.shape[0], rank, world)
    idx, s32, _ = oracle.topk(A[r0:r1], B, 7)
    i, j, s, _ = oracle.threshold(A[r0:r1], B, 0.8, want_s64=False)
    parts = shard.all_gather_object((idx, s32, i, j, s, r0))
    # contrastive: per-row loss terms and partial column logsumexps
    N, d, T = 96, 16, 0.1
    Ap, Bp = datagen.paired(N, d, 6, seed=52)
    a64, b64 = Ap.astype(np.float64), Bp.astype(np.float64)
    q0, q1 = shard.row_range(N, rank, world)
    S = a64[q0:q1] @ b64.T / T
    lse_rows = oracle.infonce_rows(a64, b64, T, np.arange(q0, q1), grads=False)[0]
    row_terms = lse_rows - np.array([S[t, q0 + t] for t in range(q1 - q0)])
    loss_part = torch.tensor([row_terms.sum()], dtype=torch.float64)
    dist.all_reduce(loss_part)
    m = S.max(axis=0)
    col_partial = m + np.log(np.exp(S - m).sum(axis=0))
    cparts = shard.all_gather_object(col_partial)
    if rank == 0:
        np.save(os.path.join(out_dir, "loss.npy"), loss_part.numpy() / N)
        np.save(os.path.join(out_dir, "lse_col.npy"), shard.lse_combine(cparts))
        import pickle
        with open(os.path.join(out_dir, "parts.pkl"), "wb") as f:
            pickle.dump(parts, f)
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_join_and_contrastive_reductions(tmp_path):
    import pickle

    import oracle
    from paper_2112_07552_gb300 import datagen, shard
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    with open(tmp_path / "parts.pkl", "rb") as f:
        parts = pickle.load(f)
    A = datagen.clustered(301, 32, 12, 0.1, seed=51, stream=0)
    B = datagen.clustered(257, 32, 12, 0.1, seed=51, stream=1)
    idx, s32 = shard.concat_topk([(p[0], p[1]) for p in parts])
    widx, ws32, _ = oracle.topk(A, B, 7)
    assert np.array_equal(idx, widx) and np.array_equal(s32.view(np.uint32), ws32.view(np.uint32))
    i, j, s = shard.concat_threshold([(p[2], p[3], p[4]) for p in parts],
                                     [p[5] for p in parts])
    wi, wj, ws, _ = oracle.threshold(A, B, 0.8, want_s64=False)
    assert np.array_equal(i, wi) and np.array_equal(j, wj) and np.array_equal(s, ws)
    N, d, T = 96, 16, 0.1
    Ap, Bp = datagen.paired(N, d, 6, seed=52)
    loss, _, lse_col, _, _ = oracle.infonce(Ap.astype(np.float64), Bp.astype(np.float64), T,
                                            sym=True, grads=False)
    # the rows' half of the symmetric loss and the combined column lse
    lse_row_loss = np.load(tmp_path / "loss.npy")[0]
    full_rows, _, _, _, _ = oracle.infonce(Ap.astype(np.float64), Bp.astype(np.float64), T,
                                           grads=False)
    assert abs(lse_row_loss - full_rows) <= 1e-12 * max(1.0, abs(full_rows))
    assert np.allclose(np.load(tmp_path / "lse_col.npy"), lse_col, rtol=1e-13, atol=1e-12)


def _infonce_worker(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_2112_07552_gb300 import datagen, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, d, T = 90, 12, 0.1
    Ap, Bp = datagen.paired(N, d, 6, seed=53)
    a64, b64 = Ap.astype(np.float64), Bp.astype(np.float64)

    # stand-ins for the library's row-shard calls: FP64, from the oracle's
    # row statistics (lse, dA rows) and the rows' dB contribution written out
    def fwd(A_rows, r0, B, T_):
        rows = np.arange(r0, r0 + A_rows.shape[0])
        lse, _ = oracle.infonce_rows(a64, b64, T_, rows, grads=True)
        S = A_rows.numpy() @ B.numpy().T / T_
        part = (lse - S[np.arange(len(rows)), rows]).sum() / N
        return torch.tensor([part], dtype=torch.float64), torch.from_numpy(lse)

    def bwd(A_rows, r0, B, T_, lse):
        rows = np.arange(r0, r0 + A_rows.shape[0])
        _, dA = oracle.infonce_rows(a64, b64, T_, rows, grads=True)
        S = A_rows.numpy() @ B.numpy().T / T_
        G = np.exp(S - lse.numpy()[:, None])
        G[np.arange(len(rows)), rows] -= 1.0
        dB = G.T @ A_rows.numpy() / (N * T_)
        return torch.from_numpy(dA), torch.from_numpy(dB)

    r0, r1 = shard.row_range(N, rank, world)
    loss, lse, dA, dB = shard.infonce_step(fwd, bwd, torch.from_numpy(a64[r0:r1]), r0,
                                           torch.from_numpy(b64), T)
    gathered = shard.all_gather_object((r0, dA.numpy()))
    if rank == 0:
        np.save(os.path.join(out_dir, "inf_loss.npy"), loss.numpy())
        np.save(os.path.join(out_dir, "inf_dB.npy"), dB.numpy())
        np.save(os.path.join(out_dir, "inf_dA.npy"),
                np.concatenate([g[1] for g in sorted(gathered, key=lambda g: g[0])]))
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_infonce_reductions(tmp_path):
    # the loss all-reduce and the dB all-reduce of shard.infonce_step over two
    # gloo ranks give the unsharded oracle's loss, dA and dB
    import oracle
    from paper_2112_07552_gb300 import datagen
    mp.spawn(_infonce_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    N, d, T = 90, 12, 0.1
    Ap, Bp = datagen.paired(N, d, 6, seed=53)
    loss, _, _, dA, dB = oracle.infonce(Ap.astype(np.float64), Bp.astype(np.float64), T)
    assert abs(np.load(tmp_path / "inf_loss.npy")[0] - loss) <= 1e-12 * max(1.0, abs(loss))
    assert np.allclose(np.load(tmp_path / "inf_dA.npy"), dA, rtol=1e-10, atol=1e-13)
    assert np.allclose(np.load(tmp_path / "inf_dB.npy"), dB, rtol=1e-10, atol=1e-13)


def test_row_range_partitions():
    from paper_2112_07552_gb300 import shard
    for n in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard.row_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
