"""Seeded synthetic inputs for the similarity join (shared by tests, bench, oracle).

This module holds no arithmetic of the join itself: it only draws embeddings.
Every array is a deterministic function of (seed, stream, shape), drawn with
NumPy's counter-based Philox generator in fixed-size row chunks, so the result
does not depend on the number of threads used.

Recipes (the workloads of the join):
  * clustered: K centres uniform on the unit sphere (normalised Gaussians);
    each row picks a centre (iid uniform, or Zipf(s) over the centre ranks),
    adds isotropic Gaussian noise whose TOTAL expected squared norm is
    sigma^2 (per-coordinate std sigma/sqrt(d)), and is renormalised in FP64
    before rounding to float32.
  * near duplicates: a seeded fraction of rows i < min(nA, nB) gets
    b_{pi(i)} = normalise(a_i + n), ||n|| ~ sigma_dup (total), pi a seeded
    permutation of B's rows.
  * one-hot / multi-attribute one-hot: the relational encoding of Sec. 3.1 of
    the paper (mat(A)_ij = 1 iff a_i.ID = v_j), optionally one block per
    attribute scaled by 1/sqrt(#attributes).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CHUNK = 8192  # rows per RNG chunk; part of the recipe (changing it changes data)


def _rng(seed: int, stream: int, chunk: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, stream, chunk])))


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _normalise_rows(x64: np.ndarray) -> np.ndarray:
    n = np.sqrt(np.einsum("ij,ij->i", x64, x64))
    n[n == 0] = 1.0
    return (x64 / n[:, None]).astype(np.float32)


def centres(n_clusters: int, d: int, seed: int) -> np.ndarray:
    """n_clusters unit vectors, uniform on the sphere (float64)."""
    out = np.empty((n_clusters, d), np.float64)
    for c0 in range(0, n_clusters, CHUNK):
        c1 = min(n_clusters, c0 + CHUNK)
        g = _rng(seed, 1000, c0 // CHUNK).standard_normal((c1 - c0, d))
        out[c0:c1] = g / np.linalg.norm(g, axis=1, keepdims=True)
    return out


def assignments(n: int, n_clusters: int, seed: int, stream: int,
                zipf_s: float | None = None) -> np.ndarray:
    """Centre index per row: iid uniform, or Zipf(zipf_s) over ranks 1..K."""
    rng = _rng(seed, 2000 + stream, 0)
    if zipf_s is None:
        return rng.integers(0, n_clusters, size=n, dtype=np.int64)
    ranks = np.arange(1, n_clusters + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** (-float(zipf_s)))
    cdf /= cdf[-1]
    u = rng.random(n)
    r = np.minimum(np.searchsorted(cdf, u, side="right"), n_clusters - 1)
    perm = _rng(seed, 3000, 0).permutation(n_clusters)  # rank -> centre id
    return perm[r]


def clustered(n: int, d: int, n_clusters: int, sigma: float = 0.1, seed: int = 0,
              stream: int = 0, zipf_s: float | None = None,
              noise_mode: str = "total", C: np.ndarray | None = None) -> np.ndarray:
    """n x d float32 unit rows drawn around shared centres (see module doc)."""
    if C is None:
        C = centres(n_clusters, d, seed)
    asg = assignments(n, n_clusters, seed, stream, zipf_s)
    if noise_mode == "total":
        std = sigma / np.sqrt(d)
    elif noise_mode == "per_coord":
        std = sigma
    else:
        raise ValueError("noise_mode must be 'total' or 'per_coord'")
    out = np.empty((n, d), np.float32)

    def work(ci):
        r0 = ci * CHUNK
        r1 = min(n, r0 + CHUNK)
        g = _rng(seed, 10 + stream, ci).standard_normal((r1 - r0, d), dtype=np.float32)
        x = C[asg[r0:r1]] + std * g.astype(np.float64)
        out[r0:r1] = _normalise_rows(x)

    nchunks = (n + CHUNK - 1) // CHUNK
    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(work, range(nchunks)))
    return out


def add_near_duplicates(A: np.ndarray, B: np.ndarray, frac: float, sigma: float,
                        seed: int = 0) -> np.ndarray:
    """Return (pairs) and overwrite rows of B with noisy copies of rows of A.

    pairs[:, 0] = i (row of A), pairs[:, 1] = pi(i) (row of B).
    """
    n = min(A.shape[0], B.shape[0])
    d = A.shape[1]
    rng = _rng(seed, 4000, 0)
    m = int(round(frac * n))
    src = np.sort(rng.choice(n, size=m, replace=False))
    perm = rng.permutation(B.shape[0])
    dst = perm[src]
    std = sigma / np.sqrt(d)
    for c0 in range(0, m, CHUNK):
        c1 = min(m, c0 + CHUNK)
        g = _rng(seed, 4001, c0 // CHUNK).standard_normal((c1 - c0, d))
        B[dst[c0:c1]] = _normalise_rows(A[src[c0:c1]].astype(np.float64) + std * g)
    return np.stack([src, dst], axis=1)


def paired(n: int, d: int, n_clusters: int, sigma: float = 0.1, sigma_pair: float = 0.02,
           seed: int = 0):
    """(A, B) with b_i a near duplicate of a_i (positives on the diagonal)."""
    A = clustered(n, d, n_clusters, sigma, seed, stream=0)
    std = sigma_pair / np.sqrt(d)
    B = np.empty_like(A)
    for c0 in range(0, n, CHUNK):
        c1 = min(n, c0 + CHUNK)
        g = _rng(seed, 5000, c0 // CHUNK).standard_normal((c1 - c0, d))
        B[c0:c1] = _normalise_rows(A[c0:c1].astype(np.float64) + std * g)
    return A, B


def one_hot(keys: np.ndarray, n_values: int) -> np.ndarray:
    """mat(X)_ij = 1 iff key_i == v_j (Sec. 3.1), float32."""
    keys = np.asarray(keys, dtype=np.int64)
    out = np.zeros((keys.shape[0], n_values), np.float32)
    out[np.arange(keys.shape[0]), keys] = 1.0
    return out


def multi_attr_one_hot(key_cols, domains) -> np.ndarray:
    """One one-hot block per attribute, each scaled by 1/sqrt(#attributes).

    With 4 attributes the scale is exactly 1/2, so <a, b> = (#equal attributes)/4.
    """
    na = len(domains)
    scale = np.float32(1.0 / np.sqrt(na))
    blocks = [one_hot(k, v) * scale for k, v in zip(key_cols, domains)]
    return np.ascontiguousarray(np.concatenate(blocks, axis=1))


def keys(n: int, n_distinct: int, seed: int, stream: int) -> np.ndarray:
    """n uniform keys in [0, n_distinct)."""
    return _rng(seed, 6000 + stream, 0).integers(0, n_distinct, size=n, dtype=np.int64)


def unit_rows(n: int, d: int, seed: int, stream: int) -> np.ndarray:
    """n iid uniform unit vectors (float32)."""
    out = np.empty((n, d), np.float32)
    for c0 in range(0, n, CHUNK):
        c1 = min(n, c0 + CHUNK)
        out[c0:c1] = _normalise_rows(_rng(seed, 7000 + stream, c0 // CHUNK)
                                     .standard_normal((c1 - c0, d)))
    return out


def log_uniform_sizes(n_jobs: int, lo: int, hi: int, seed: int, stream: int) -> np.ndarray:
    """Integer sizes log-uniform in [lo, hi]."""
    u = _rng(seed, 8000 + stream, 0).random(n_jobs)
    return np.minimum(hi, np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo))))
                      ).astype(np.int64)


def batch_centre_counts(sizes_a: np.ndarray, sizes_b: np.ndarray) -> np.ndarray:
    """Centres per job of an uneven batch: max(1, max(nA, nB) // 10)."""
    return np.maximum(1, np.maximum(sizes_a, sizes_b) // 10).astype(np.int64)


def clustered_batch_device(sizes_a, sizes_b, d: int, sigma: float = 0.1, seed: int = 0,
                           device="cuda", chunk_rows: int = 1 << 20):
    """An uneven batch of clustered joins drawn on a torch device.

    Job q has K_q = max(1, max(nA_q, nB_q) // 10) centres uniform on the unit
    sphere, shared by its A and B; every row picks one of its job's centres
    iid uniformly, adds isotropic Gaussian noise of total expected squared
    norm sigma^2 (per-coordinate std sigma / sqrt(d)) and is renormalised in
    float64 before rounding to float32.  Draws come from torch's Philox
    generator on the device, seeded with `seed`, in a fixed order (centres,
    then A rows, then B rows, chunk_rows rows at a time), so the arrays are a
    deterministic function of (sizes, d, sigma, seed, chunk_rows) for a given
    torch build.  (Batches of tens of millions of rows are out of reach of the
    host generator within a benchmark's time.)

    Returns (A, B, a_off, b_off): float32 device tensors holding every job's
    rows back to back, and the row offsets of the jobs (int64, n_jobs + 1).
    """
    import torch

    sizes_a = np.asarray(sizes_a, np.int64)
    sizes_b = np.asarray(sizes_b, np.int64)
    n_jobs = len(sizes_a)
    K = batch_centre_counts(sizes_a, sizes_b)
    c_off = np.concatenate([[0], np.cumsum(K)])
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    C = torch.empty((int(c_off[-1]), d), dtype=torch.float32, device=device)
    for c0 in range(0, C.shape[0], chunk_rows):
        c1 = min(C.shape[0], c0 + chunk_rows)
        x = torch.randn((c1 - c0, d), generator=g, dtype=torch.float64, device=device)
        C[c0:c1] = (x / x.norm(dim=1, keepdim=True)).float()
    Kd = torch.from_numpy(K).to(device)
    cod = torch.from_numpy(c_off[:-1]).to(device)

    def side(sizes):
        off = np.concatenate([[0], np.cumsum(sizes)])
        X = torch.empty((int(off[-1]), d), dtype=torch.float32, device=device)
        job = torch.from_numpy(np.repeat(np.arange(n_jobs, dtype=np.int64), sizes)).to(device)
        for r0 in range(0, X.shape[0], chunk_rows):
            r1 = min(X.shape[0], r0 + chunk_rows)
            jr = job[r0:r1]
            u = torch.rand(r1 - r0, generator=g, dtype=torch.float64, device=device)
            local = torch.minimum((u * Kd[jr]).long(), Kd[jr] - 1)
            x = C[cod[jr] + local].double()
            x += torch.randn((r1 - r0, d), generator=g, dtype=torch.float64,
                             device=device) * (sigma / np.sqrt(d))
            X[r0:r1] = (x / x.norm(dim=1, keepdim=True)).float()
        return X, off

    A, a_off = side(sizes_a)
    B, b_off = side(sizes_b)
    del C
    return A, B, a_off, b_off


ADVERSARIAL_KINDS = ("cancel_run", "cancel_half", "spread", "alternating")


def adversarial(n: int, d: int, kind: str, seed: int = 0, side: int = 0) -> np.ndarray:
    """n x d float32 unit rows built so that many products <a_i, b_j> of an
    A side (side=0) and a B side (side=1) cancel: large partial sums and a
    small result, the hardest case for a long low-precision accumulation.

    * cancel_run: a long run of small same-sign entries and one large entry
      (at one of 8 positions) holding half the squared norm; on the B side the
      large entry has the opposite sign, so run and large term cancel.
    * cancel_half: entries of one magnitude pattern; B rows negate the second
      half of the coordinates, so the first half's sum (~ +1/2) is cancelled
      by the second half.
    * spread: magnitudes 2^-U(0, 20) with random signs (exponents across the
      whole bfloat16/E4M3 range at unit norm).
    * alternating: a_k of alternating sign against all-positive b_k.
    Every row gets a small multiplicative jitter so that no two entries are
    equal, then is normalised in FP64 and rounded to float32.
    """
    if kind not in ADVERSARIAL_KINDS:
        raise ValueError("unknown kind %r" % kind)
    rng = _rng(seed, 5000 + 10 * ADVERSARIAL_KINDS.index(kind) + side, 0)
    jit = 1.0 + 0.05 * rng.standard_normal((n, d))
    if kind == "cancel_run":
        x = np.full((n, d), 1.0 / np.sqrt(2.0 * (d - 1)))
        pos = rng.integers(0, 8, size=n) * (d // 8) + (d // 8 - 1)
        big = np.sqrt(0.5) * (-1.0 if side else 1.0)
        x[np.arange(n), pos] = big
    elif kind == "cancel_half":
        base = _rng(seed, 5099, 0).uniform(0.5, 1.5, size=d)
        x = np.tile(base, (n, 1))
        if side:
            x[:, d // 2:] *= -1.0
    elif kind == "spread":
        e = rng.uniform(0.0, 20.0, size=(n, d))
        s = rng.choice([-1.0, 1.0], size=(n, d))
        x = s * np.exp2(-e)
    else:  # alternating
        x = rng.uniform(0.5, 1.5, size=(n, d))
        if side == 0:
            x[:, 1::2] *= -1.0
    return _normalise_rows(x * jit)
