"""Host-side logic of the multi-GPU join (one process per GPU).

The join shards by rows of A with B replicated: every left row's top-k and
threshold set depend on that row alone, so ranks exchange nothing while
joining.  Results are concatenated with global row offsets.  The contrastive
join, sharded the same way, needs two reductions: the loss is a sum of
per-row terms (all-reduce of one value) and the gradient of B a sum of the
rows' contributions (all-reduce of N x d values); the symmetric variant's
column logsumexp would combine per-rank partial column logsumexps
(logsumexp over ranks, lse_combine).
"""
from __future__ import annotations

import numpy as np


def row_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced row range [r0, r1) of `rank` among `world` ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def concat_topk(parts):
    """Row-sharded top-k results [(idx, score), ...] in rank order -> full arrays."""
    return (np.concatenate([p[0] for p in parts], axis=0),
            np.concatenate([p[1] for p in parts], axis=0))


def concat_threshold(parts, row_starts):
    """Row-sharded threshold pairs [(i_local, j, score), ...] -> global (i, j, score).

    Each part is sorted by (i, j) within its shard; shards are in rank order, so
    the concatenation is sorted by (i, j) globally.
    """
    i = np.concatenate([np.asarray(p[0]) + r0 for p, r0 in zip(parts, row_starts)])
    j = np.concatenate([np.asarray(p[1]) for p in parts])
    s = np.concatenate([np.asarray(p[2]) for p in parts])
    return i, j, s


def lse_combine(partials) -> np.ndarray:
    """logsumexp over ranks of per-rank partial logsumexps (elementwise)."""
    P = np.stack([np.asarray(p, dtype=np.float64) for p in partials])
    m = np.max(P, axis=0)
    with np.errstate(invalid="ignore"):
        out = m + np.log(np.sum(np.exp(P - m), axis=0))
    return np.where(np.isneginf(m), -np.inf, out)


def all_gather_object(obj, group=None):
    """torch.distributed all_gather_object wrapper (rank order)."""
    import torch.distributed as dist
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, obj, group=group)
    return out


def infonce_step(fwd_rows, bwd_rows, A_rows, r0: int, B, T: float, group=None):
    """One row-sharded contrastive step on this rank: forward and backward of
    rows [r0, r0 + n) against all of B, then the two reductions over the
    ranks (torch.distributed, when initialised): the loss (sum of the ranks'
    parts) and dB (sum of the ranks' contributions).  fwd_rows(A_rows, r0, B,
    T) -> (loss_part [1], lse_rows) and bwd_rows(A_rows, r0, B, T, lse_rows)
    -> (dA_rows, dB_part) are the library's row-shard calls (see
    library_rows).  Returns (loss, lse_rows, dA_rows, dB); loss and dB are
    the same on every rank."""
    import torch.distributed as dist
    loss_part, lse = fwd_rows(A_rows, r0, B, T)
    dA, dB = bwd_rows(A_rows, r0, B, T, lse)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(loss_part, group=group)
        dist.all_reduce(dB, group=group)
    return loss_part, lse, dA, dB


def library_rows(J):
    """(fwd_rows, bwd_rows) of infonce_step through a SimilarityJoin handle
    (sj_contrastive_fwd_rows / sj_backward_rows, upstream gradient 1)."""
    import torch

    def fwd(A_rows, r0, B, T):
        return J.contrastive_forward_rows(A_rows, r0, B, T)

    def bwd(A_rows, r0, B, T, lse):
        return J.contrastive_backward_rows(A_rows, r0, B, T, lse,
                                           torch.ones(1, device=A_rows.device))
    return fwd, bwd
