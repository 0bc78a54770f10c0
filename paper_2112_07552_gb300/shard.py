"""Host-side logic of the multi-GPU join (one process per GPU).

The join shards by rows of A with B replicated: every left row's top-k and
threshold set depend on that row alone, so ranks exchange nothing while
joining.  Results are concatenated with global row offsets.  The contrastive
join, sharded the same way, needs two reductions: the loss is a sum of
per-row terms (all-reduce), and the symmetric variant's column logsumexp
combines per-rank partial column logsumexps (logsumexp over ranks).
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
