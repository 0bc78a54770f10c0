"""Oracle for the paper's relational join patterns (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
use this module; nothing in the product path imports it.  It shares no code
with the CUDA library.

Definitions written out (Sec. 3.1 "Two-way natural join" and Sec. 3.3
"Group-by aggregates over joins"):

* block(ka, kb, min_match): rows of A and B carry n_attr key attributes.
  mat(A) has one one-hot block per attribute, scaled by c = fl32(1/sqrt(n_attr))
  (so every row has unit norm); C = mat(A) mat(B)^T.  C_ij = (number of equal
  attributes of a_i and b_j) * c^2 exactly.  The join keeps (i, j) when at
  least min_match attributes are equal (for n_attr = 1 and min_match = 1: the
  equi-join Q1, C_ij > 0), ordered by (i, j), with score RN_fp32(C_ij).
* groupby_sum (Q3): SELECT B.G, SUM(A.Val), COUNT(*) FROM A, B
  WHERE A.ID = B.ID GROUP BY B.G -- every pair of the join counts (bag
  semantics; the paper's 0/1 mat(B) gives the same result when B holds no
  duplicate (ID, G) tuple), groups ordered by value, exact integer sums.
* sum_product (Q4): SELECT SUM(A.Val * B.Val), COUNT(*) FROM A, B
  WHERE A.ID = B.ID, exact integers.
"""
from __future__ import annotations

import numpy as np


def _pairs_equal(ka: np.ndarray, kb: np.ndarray):
    """All (i, j) with ka[i] == kb[j]: sort B's keys, then for each A key the
    run of equal B keys (a sort and a binary search as library steps)."""
    ka = np.asarray(ka, np.int64)
    kb = np.asarray(kb, np.int64)
    order = np.argsort(kb, kind="stable")
    sk = kb[order]
    lo = np.searchsorted(sk, ka, side="left")
    hi = np.searchsorted(sk, ka, side="right")
    cnt = hi - lo
    i = np.repeat(np.arange(ka.shape[0], dtype=np.int64), cnt)
    starts = np.repeat(lo, cnt)
    within = np.arange(i.shape[0], dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    j = order[starts + within]
    return i, j


def block(ka, kb, min_match: int = 1):
    """(i, j, score float32) of every pair agreeing on >= min_match of the
    n_attr key attributes (columns of ka, kb), sorted by (i, j)."""
    ka = np.asarray(ka, np.int64)
    kb = np.asarray(kb, np.int64)
    if ka.ndim == 1:
        ka, kb = ka[:, None], kb[:, None]
    n_attr = ka.shape[1]
    nB = kb.shape[0]
    # every (pair, attribute) with equal values, as the pair's index i * nB + j;
    # a pair's number of equal attributes is how often its index occurs
    per_attr = []
    for a in range(n_attr):
        i, j = _pairs_equal(ka[:, a], kb[:, a])
        per_attr.append(i * nB + j)
    allk = np.concatenate(per_attr) if per_attr else np.zeros(0, np.int64)
    u, cnt = np.unique(allk, return_counts=True)
    keys, m = u[cnt >= min_match], cnt[cnt >= min_match].astype(np.int64)
    c = float(np.float32(1.0 / np.sqrt(n_attr)))
    s64 = m.astype(np.float64) * (c * c)  # exact: a 48-bit square times a small count
    return keys // max(nB, 1), keys % max(nB, 1), s64.astype(np.float32)


def groupby_sum(a_id, a_val, b_id, b_group):
    """Q3: [(group, SUM(A.Val), COUNT(*))] over the join A.ID = B.ID, by group."""
    sums, cnts = {}, {}
    for k, v in zip(np.asarray(a_id).tolist(), np.asarray(a_val).tolist()):
        sums[k] = sums.get(k, 0) + int(v)
        cnts[k] = cnts.get(k, 0) + 1
    gs, gc = {}, {}
    for k, g in zip(np.asarray(b_id).tolist(), np.asarray(b_group).tolist()):
        if k in cnts:
            gs[g] = gs.get(g, 0) + sums[k]
            gc[g] = gc.get(g, 0) + cnts[k]
    return [(g, gs[g], gc[g]) for g in sorted(gc)]


def sum_product(a_id, a_val, b_id, b_val):
    """Q4: (SUM(A.Val * B.Val), COUNT(*)) over the join A.ID = B.ID."""
    sums, cnts = {}, {}
    for k, v in zip(np.asarray(a_id).tolist(), np.asarray(a_val).tolist()):
        sums[k] = sums.get(k, 0) + int(v)
        cnts[k] = cnts.get(k, 0) + 1
    tot, cnt = 0, 0
    for k, v in zip(np.asarray(b_id).tolist(), np.asarray(b_val).tolist()):
        if k in cnts:
            tot += sums[k] * int(v)
            cnt += cnts[k]
    return tot, cnt
