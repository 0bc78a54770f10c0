"""GPU parity: the CUDA join through the C ABI against the oracle.

The bar is exact: identical index sets and orders, and bit-identical float32
scores (each the round-to-nearest-even of the exact dot product), for both the
tensor-core (bf16) and the plain FP32 scoring pass.
"""
import numpy as np
import pytest

import oracle
from paper_2112_07552_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ("bf16", "fp32", "fp8", "bf16x3")


@pytest.fixture(scope="module")
def sjmod():
    from paper_2112_07552_gb300 import _build, sj
    _build.build()
    return sj


_handles = {}


def join(sjmod, d, prec):
    key = (d, prec)
    if key not in _handles:
        _handles[key] = sjmod.SimilarityJoin(d, prec=prec, device=0)
    return _handles[key]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def assert_topk(got_idx, got_s, A, B, k, rows=None):
    idx, s32, _ = oracle.topk(A, B, k, rows=rows)
    gi = got_idx.cpu().numpy() if hasattr(got_idx, "cpu") else got_idx
    gs = got_s.cpu().numpy() if hasattr(got_s, "cpu") else got_s
    if rows is not None:
        gi, gs = gi[rows], gs[rows]
    bad = np.nonzero((gi != idx).any(axis=1) | (gs.view(np.uint32) != s32.view(np.uint32)).any(axis=1))[0]
    assert bad.size == 0, "rows %s differ: got %s %s want %s %s" % (
        bad[:5], gi[bad[:1]], gs[bad[:1]], idx[bad[:1]], s32[bad[:1]])


def assert_thr(got, A, B, tau):
    gi, gj, gs = [t.cpu().numpy() for t in got]
    wi, wj, ws, _ = oracle.threshold(A, B, tau, want_s64=False)
    assert gi.shape == wi.shape, (gi.shape, wi.shape)
    assert np.array_equal(gi, wi) and np.array_equal(gj, wj)
    assert np.array_equal(gs.view(np.uint32), ws.view(np.uint32))


@pytest.mark.parametrize("prec", PRECS)
def test_fp32_config_full(sjmod, prec):
    # 2,000 x 2,000, d = 256, 200 clusters, sigma = 0.1, k = 10, tau = 0.8, seed 0
    A = datagen.clustered(2000, 256, 200, 0.1, seed=0, stream=0)
    B = datagen.clustered(2000, 256, 200, 0.1, seed=0, stream=1)
    J = join(sjmod, 256, prec)
    idx, sc = J.topk(dev(A), dev(B), 10)
    assert_topk(idx, sc, A, B, 10)
    assert_thr(J.threshold(dev(A), dev(B), 0.8), A, B, 0.8)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nA,nB,d", [(1, 1, 1), (1, 300, 3), (127, 129, 100), (129, 257, 64),
                                     (255, 511, 257), (300, 1000, 33), (513, 700, 128)])
def test_ragged_sizes(sjmod, prec, nA, nB, d):
    A = datagen.clustered(nA, d, max(1, nA // 10), 0.2, seed=3, stream=0)
    B = datagen.clustered(nB, d, max(1, nA // 10), 0.2, seed=3, stream=1)
    J = join(sjmod, d, prec)
    for k in (1, 5, 37):
        idx, sc = J.topk(dev(A), dev(B), k)
        assert_topk(idx, sc, A, B, k)
    for tau in (0.0, 0.5, 0.9):
        assert_thr(J.threshold(dev(A), dev(B), tau), A, B, tau)


@pytest.mark.parametrize("prec", PRECS)
def test_k_larger_than_B_pads(sjmod, prec):
    A = datagen.unit_rows(40, 16, 1, 0)
    B = datagen.unit_rows(6, 16, 1, 1)
    J = join(sjmod, 16, prec)
    idx, sc = J.topk(dev(A), dev(B), 9)
    assert_topk(idx, sc, A, B, 9)
    assert (idx[:, 6:] == -1).all() and torch.isinf(sc[:, 6:]).all()


@pytest.mark.parametrize("prec", PRECS)
def test_self_join_invariants(sjmod, prec):
    X = datagen.clustered(700, 64, 30, 0.1, seed=4)
    J = join(sjmod, 64, prec)
    dX = dev(X)
    idx, sc = J.topk(dX, dX, 12)
    assert_topk(idx, sc, X, X, 12)
    # own top-1
    top1 = idx[:, 0].cpu().numpy()
    assert np.all(top1 <= np.arange(700))
    i, j, s = J.threshold(dX, dX, 0.9)
    assert_thr((i, j, s), X, X, 0.9)
    # symmetry of the pair set
    pairs = set(zip(i.cpu().tolist(), j.cpu().tolist()))
    assert all((b, a) in pairs for a, b in pairs)


@pytest.mark.parametrize("prec", PRECS)
def test_exact_ties_duplicates_and_onehot(sjmod, prec):
    # one-hot rows (Sec. 3.1): scores exactly 0/1, massive exact ties
    ka = datagen.keys(300, 12, 0, 0)
    kb = datagen.keys(900, 12, 0, 1)
    A, B = datagen.one_hot(ka, 12), datagen.one_hot(kb, 12)
    J = join(sjmod, 12, prec)
    idx, sc = J.topk(dev(A), dev(B), 10)
    assert_topk(idx, sc, A, B, 10)
    assert_thr(J.threshold(dev(A), dev(B), 1.0), A, B, 1.0)
    assert_thr(J.threshold(dev(A), dev(B), 2.0 ** -30), A, B, 2.0 ** -30)
    # duplicated rows in B
    X = datagen.unit_rows(64, 40, 5, 0)
    Y = np.repeat(datagen.unit_rows(50, 40, 5, 1), 3, axis=0)
    J2 = join(sjmod, 40, prec)
    idx, sc = J2.topk(dev(X), dev(Y), 8)
    assert_topk(idx, sc, X, Y, 8)


@pytest.mark.parametrize("prec", PRECS)
def test_hadamard_and_inclusive_tau(sjmod, prec):
    H = np.array([[1.0]])
    while H.shape[0] < 256:
        H = np.block([[H, H], [H, -H]])
    H = (H / 16.0).astype(np.float32)
    A, B = H[:100], np.concatenate([H[50:200], -H[:30]])
    J = join(sjmod, 256, prec)
    idx, sc = J.topk(dev(A), dev(B), 4)
    assert_topk(idx, sc, A, B, 4)
    for tau in (1.0, 0.0, -1.0):
        assert_thr(J.threshold(dev(A), dev(B), tau), A, B, tau)


@pytest.mark.parametrize("prec", PRECS)
def test_host_pointers(sjmod, prec):
    A = datagen.clustered(333, 48, 20, 0.1, seed=6, stream=0)
    B = datagen.clustered(444, 48, 20, 0.1, seed=6, stream=1)
    J = join(sjmod, 48, prec)
    idx, sc = J.topk(torch.from_numpy(A), torch.from_numpy(B), 6)
    assert idx.device.type == "cpu"
    assert_topk(idx, sc, A, B, 6)
    assert_thr(J.threshold(torch.from_numpy(A), torch.from_numpy(B), 0.7), A, B, 0.7)


@pytest.mark.parametrize("prec", PRECS)
def test_validation_errors(sjmod, prec):
    J = join(sjmod, 8, prec)
    A = datagen.unit_rows(10, 8, 0, 0)
    bad = A.copy()
    bad[3, 2] = np.nan
    with pytest.raises(sjmod.SJError) as e:
        J.topk(dev(bad), dev(A), 2)
    assert e.value.code == sjmod.SJ_ERR_NONFINITE
    bad = A.copy()
    bad[1] *= 1.01
    with pytest.raises(sjmod.SJError) as e:
        J.threshold(dev(A), dev(bad), 0.5)
    assert e.value.code == sjmod.SJ_ERR_NOT_UNIT_NORM
    # the handle stays usable
    idx, sc = J.topk(dev(A), dev(A), 3)
    assert_topk(idx, sc, A, A, 3)


@pytest.mark.parametrize("prec", PRECS)
def test_capacity_reports_required_count(sjmod, prec):
    import ctypes
    A = datagen.clustered(200, 32, 5, 0.1, seed=8, stream=0)
    B = datagen.clustered(300, 32, 5, 0.1, seed=8, stream=1)
    wi, _, _, _ = oracle.threshold(A, B, 0.5, want_s64=False)
    assert len(wi) > 10
    J = join(sjmod, 32, prec)
    out = torch.empty((10, 3), dtype=torch.int64, device="cuda")
    n = sjmod.I64(0)
    dA, dB = dev(A), dev(B)  # keep both alive for the duration of the call
    code = sjmod.lib().sj_threshold(J.handle, dA.data_ptr(), 200, dB.data_ptr(), 300,
                                    0.5, out.data_ptr(), 10, ctypes.byref(n), None)
    assert code == sjmod.SJ_ERR_CAPACITY and n.value == len(wi)


def test_empty_inputs(sjmod):
    J = join(sjmod, 8, "bf16")
    A = datagen.unit_rows(5, 8, 0, 0)
    E = np.zeros((0, 8), np.float32)
    idx, sc = J.topk(dev(A), dev(E), 3)
    assert (idx == -1).all() and torch.isinf(sc).all()
    idx, sc = J.topk(dev(E), dev(A), 3)
    assert idx.shape == (0, 3)
    i, j, s = J.threshold(dev(A), dev(E), 0.1)
    assert i.numel() == 0


def test_debug_timeout_returns_status_and_context_survives(sjmod):
    J = sjmod.SimilarityJoin(64, prec="bf16", device=0, flags=sjmod.SJ_FLAG_DEBUG_TIMEOUT)
    A = datagen.unit_rows(300, 64, 0, 0)
    with pytest.raises(sjmod.SJError) as e:
        J.topk(dev(A), dev(A), 4)
    assert e.value.code == sjmod.SJ_ERR_TIMEOUT
    J.close()
    # the context is still usable afterwards
    J2 = join(sjmod, 64, "bf16")
    idx, sc = J2.topk(dev(A), dev(A), 4)
    assert_topk(idx, sc, A, A, 4)


def test_batch_matches_single_calls(sjmod):
    J = join(sjmod, 64, "bf16")
    jobs, data = [], []
    for q, (na, nb) in enumerate([(100, 150), (1, 700), (300, 20), (257, 257)]):
        A = datagen.clustered(na, 64, 10, 0.1, seed=20 + q, stream=0)
        B = datagen.clustered(nb, 64, 10, 0.1, seed=20 + q, stream=1)
        data.append((A, B))
        jobs.append({"A": dev(A), "B": dev(B), "k": 5, "tau": 0.8})
    outs = J.batch(jobs)
    for (A, B), o in zip(data, outs):
        assert_topk(o["idx"], o["score"], A, B, 5)
        assert_thr((o["i"], o["j"], o["pair_score"]), A, B, 0.8)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nA,nB,keys,k", [
    (50, 1300, 2, 10),   # ~650 exact ties per row: band overflow -> rescan -> shared-memory rank
    (20, 3000, 2, 10),   # ~1500 ties: global-memory ranker
    (8, 9000, 1, 5),     # 9000 ties: rescan list cut at 4096 -> redo with full capacity
])
def test_fallback_paths_massive_ties(sjmod, prec, nA, nB, keys, k):
    ka = datagen.keys(nA, keys, 9, 0)
    kb = datagen.keys(nB, keys, 9, 1)
    A, B = datagen.one_hot(ka, keys), datagen.one_hot(kb, keys)
    # one column split: each row's candidates go through one band list
    J = sjmod.SimilarityJoin(keys, prec=prec, device=0, flags=sjmod.SJ_FLAG_SINGLE_SPLIT)
    idx, sc, st = J.topk(dev(A), dev(B), k, with_stats=True)
    J.close()
    assert_topk(idx, sc, A, B, k)
    assert st["n_overflow_rows"] > 0


def _rows_or_empty(n, d, K, seed, stream):
    if n == 0:
        return np.zeros((0, d), np.float32)
    return datagen.clustered(int(n), d, K, 0.1, seed=seed, stream=stream)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_uneven_mixed_jobs(sjmod, prec):
    """One pipeline over many uneven jobs: sizes log-uniform in [1, 2500] per
    side plus empty sides, top-k only / threshold only / both, k on both sides
    of the shared-memory heap limit, self-joins sharing one packed segment,
    host-pointer jobs and one job whose pairs exceed its first capacity."""
    d, n_jobs = 64, 48
    sa = datagen.log_uniform_sizes(n_jobs, 1, 2500, seed=5, stream=0)
    sb = datagen.log_uniform_sizes(n_jobs, 1, 2500, seed=5, stream=1)
    sa[3], sb[7], sa[11], sb[11] = 0, 0, 0, 0
    J = join(sjmod, d, prec)
    jobs, data = [], []
    for q in range(n_jobs):
        A = _rows_or_empty(sa[q], d, 12, 100 + q, 0)
        self_join = q % 9 == 4
        B = A if self_join else _rows_or_empty(sb[q], d, 12, 100 + q, 1)
        host = q % 7 == 2
        tA = torch.from_numpy(A) if host else dev(A)
        tB = tA if self_join else (torch.from_numpy(B) if host else dev(B))
        jb = {"A": tA, "B": tB}
        mode = q % 3
        k = (1, 5, 20, 40, 64)[q % 5]
        tau = (0.8, 0.6, 0.9)[q % 3]
        if mode in (0, 2):
            jb["k"] = k
        if mode in (1, 2):
            jb["tau"] = tau
            if q == 10:
                jb["capacity"] = 1  # forces the capacity retry of this job only
        jobs.append(jb)
        data.append((A, B, jb.get("k"), jb.get("tau")))
    outs, st = J.batch(jobs, with_stats=True)
    assert st["n_launches"] > 0
    for q, ((A, B, k, tau), o) in enumerate(zip(data, outs)):
        if k:
            if A.shape[0] == 0:
                assert o["idx"].shape == (0, k)
            else:
                assert_topk(o["idx"], o["score"], A, B, k)
        if tau is not None:
            assert_thr((o["i"], o["j"], o["pair_score"]), A, B, tau)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_fallback_rows_in_several_jobs(sjmod, prec):
    """Band-list overflow in two jobs of one batch: the fallback rows are
    grouped per job and rescanned against that job's B only."""
    keys = 2
    J = sjmod.SimilarityJoin(keys, prec=prec, device=0, flags=sjmod.SJ_FLAG_SINGLE_SPLIT)
    jobs, data = [], []
    for q, (nA, nB) in enumerate([(30, 1300), (7, 50), (20, 3000), (1, 1)]):
        A = datagen.one_hot(datagen.keys(nA, keys, 40 + q, 0), keys)
        B = datagen.one_hot(datagen.keys(nB, keys, 40 + q, 1), keys)
        jobs.append({"A": dev(A), "B": dev(B), "k": 10})
        data.append((A, B))
    outs, st = J.batch(jobs, with_stats=True)
    J.close()
    for (A, B), o in zip(data, outs):
        assert_topk(o["idx"], o["score"], A, B, 10)
    assert st["n_overflow_rows"] > 0


@pytest.mark.parametrize("prec", ("bf16", "fp32"))
def test_batch_split_into_groups_under_workspace_limit(sjmod, prec):
    """A batch whose workspace exceeds the handle's limit runs as several
    groups (halved by rows until each fits); results are unchanged."""
    d = 64
    sizes = [(900, 700), (40, 1200), (1500, 300), (600, 600), (1, 2000), (800, 900)]
    data = [(datagen.clustered(na, d, 12, 0.1, seed=300 + q, stream=0),
             datagen.clustered(nb, d, 12, 0.1, seed=300 + q, stream=1))
            for q, (na, nb) in enumerate(sizes)]
    jobs = [{"A": dev(A), "B": dev(B), "k": 7, "tau": 0.85} for A, B in data]
    J_all = sjmod.SimilarityJoin(d, prec=prec, device=0)
    _, st_all = J_all.batch(jobs, with_stats=True)
    J_all.close()
    # the whole batch needs about 15 MB of workspace in bf16 and 50 MB in fp32
    # (wider band lists); these limits force a split yet fit every single job
    limit = (12 << 20) if prec == "bf16" else (32 << 20)
    J = sjmod.SimilarityJoin(d, prec=prec, device=0, workspace_limit=limit)
    outs, st = J.batch(jobs, with_stats=True)
    J.close()
    for (A, B), o in zip(data, outs):
        assert_topk(o["idx"], o["score"], A, B, 7)
        assert_thr((o["i"], o["j"], o["pair_score"]), A, B, 0.85)
    assert st["n_launches"] > st_all["n_launches"]


@pytest.mark.parametrize("prec", PRECS)
def test_batch_graph_replay_new_data_and_outputs(sjmod, prec):
    """A batch of device jobs is captured as a CUDA graph on its first call and
    replayed on later calls of the same shapes, with new inputs and new output
    buffers each time (they travel in the job table, not in the graph)."""
    d = 48
    sizes = [(300, 500), (1, 900), (700, 64), (257, 257)]
    J = sjmod.SimilarityJoin(d, prec=prec, device=0)
    replayed = []
    for call in range(3):
        data = [(datagen.clustered(na, d, 9, 0.1, seed=500 + 10 * call + q, stream=0),
                 datagen.clustered(nb, d, 9, 0.1, seed=500 + 10 * call + q, stream=1))
                for q, (na, nb) in enumerate(sizes)]
        jobs = [{"A": dev(A), "B": dev(B), "k": 6, "tau": 0.8} for A, B in data]
        outs, st = J.batch(jobs, with_stats=True)
        replayed.append(st["graph_replayed"])
        for (A, B), o in zip(data, outs):
            assert_topk(o["idx"], o["score"], A, B, 6)
            assert_thr((o["i"], o["j"], o["pair_score"]), A, B, 0.8)
    J.close()
    assert replayed[1] >= 1 and replayed[2] >= 1  # the wrapper may retry for capacity
    # a validation error inside a replayed graph is still reported
    A = datagen.clustered(300, d, 9, 0.1, seed=1, stream=0)
    B = datagen.clustered(500, d, 9, 0.1, seed=1, stream=1)
    J = sjmod.SimilarityJoin(d, prec=prec, device=0)
    J.topk(dev(A), dev(B), 6)
    bad = A.copy()
    bad[5, 3] = np.nan
    with pytest.raises(sjmod.SJError) as ei:
        J.topk(dev(bad), dev(B), 6)
    assert ei.value.code == sjmod.SJ_ERR_NONFINITE
    idx, sc = J.topk(dev(A), dev(B), 6)
    assert_topk(idx, sc, A, B, 6)
    J.close()
    # SJ_FLAG_NO_GRAPH: launches only
    J = sjmod.SimilarityJoin(d, prec=prec, device=0, flags=sjmod.SJ_FLAG_NO_GRAPH)
    for _ in range(2):
        _, _, st = J.topk(dev(A), dev(B), 6, with_stats=True)
        assert st["graph_replayed"] == 0
    J.close()


@pytest.mark.parametrize("nA,nB", [(300, 60), (129, 128), (257, 129), (700, 1000), (65, 2049)])
def test_narrow_tiles_parity(sjmod, nA, nB):
    """128-column score tiles (the tile shape the autotuner may pick) give the
    same exact results; padded work counts 128 x 128 tiles."""
    d, k, tau = 64, 7, 0.8
    A = datagen.clustered(nA, d, 11, 0.1, seed=nA, stream=0)
    B = datagen.clustered(nB, d, 11, 0.1, seed=nB, stream=1)
    J = sjmod.SimilarityJoin(d, prec="bf16", device=0, flags=sjmod.SJ_FLAG_NARROW_TILES)
    outs, st = J.batch([{"A": dev(A), "B": dev(B), "k": k, "tau": tau}], with_stats=True)
    J.close()
    o = outs[0]
    assert_topk(o["idx"], o["score"], A, B, k)
    assert_thr((o["i"], o["j"], o["pair_score"]), A, B, tau)
    padded = (-(-nA // 128) * 128) * (-(-nB // 128) * 128)
    assert st["padded_pair_scores"] == padded


def test_autotune_table_round_trip(sjmod, tmp_path):
    """sj_autotune times both tile widths per size class, writes the table,
    and a new handle that loads it joins exactly."""
    d, k = 64, 5
    path = str(tmp_path / "tiles.txt")
    J = sjmod.SimilarityJoin(d, prec="bf16", device=0)
    J.autotune(k, path)
    J.close()
    rows = [tuple(int(x) for x in line.split()) for line in open(path)]
    assert len(rows) == 11
    assert all(r[0] == d and r[1] == 1 and r[2] == k and r[4] in (128, 256) for r in rows)
    assert sorted(r[3] for r in rows) == list(range(6, 17))
    J = sjmod.SimilarityJoin(d, prec="bf16", device=0)
    J.autotune_load(path)
    for nA, nB in [(200, 100), (333, 700), (90, 5000)]:
        A = datagen.clustered(nA, d, 11, 0.1, seed=nA + 7, stream=0)
        B = datagen.clustered(nB, d, 11, 0.1, seed=nB + 7, stream=1)
        idx, sc = J.topk(dev(A), dev(B), k)
        assert_topk(idx, sc, A, B, k)
    J.close()


def _e4m3_exponent(mx):
    """Largest e with mx 2^e <= 448 (as the packing does)."""
    f, E = np.frexp(mx)
    return np.where(f <= 0.875, 9 - E, 8 - E)


def test_fp8_scores_within_their_bound(sjmod):
    """E4M3 scoring: the largest |s~ - s| over the rescored candidates stays
    within the quantisation error (recomputed here from E4M3 rounding of the
    scaled rows) plus the accumulation allowance (d + 32) 2^-13."""
    nA, nB, d, k = 600, 2500, 256, 20
    A = datagen.clustered(nA, d, 50, 0.1, seed=71, stream=0)
    B = datagen.clustered(nB, d, 50, 0.1, seed=71, stream=1)
    J = sjmod.SimilarityJoin(d, prec="fp8", device=0)
    idx, sc, st = J.topk(dev(A), dev(B), k, with_stats=True)
    J.close()
    assert_topk(idx, sc, A, B, k)
    eA = _e4m3_exponent(np.abs(A).max(axis=1))[:, None].astype(np.float64)
    eB = float(_e4m3_exponent(np.abs(B).max()))
    qa = (torch.from_numpy(A.astype(np.float64) * 2.0 ** eA).float()
          .to(torch.float8_e4m3fn).double().numpy()) * 2.0 ** -eA
    qb = (torch.from_numpy(B.astype(np.float64) * 2.0 ** eB).float()
          .to(torch.float8_e4m3fn).double().numpy()) * 2.0 ** -eB
    quant = np.abs(qa @ qb.T - A.astype(np.float64) @ B.astype(np.float64).T).max()
    acc = (d + 32) * 2.0 ** -13 * np.linalg.norm(qa, axis=1).max() * np.linalg.norm(qb, axis=1).max()
    assert 0 < st["max_abs_err_lowprec"] <= quant + acc
    # the proven per-row margin bounds every pair's quantisation error and
    # every observed error (it also carries the accumulation allowance)
    assert st["margin_max"] >= quant and st["margin_max"] >= st["max_abs_err_lowprec"]


def test_bf16x3_narrows_dense_bands(sjmod):
    """One dense cluster (cosines near 0.99 with a spread near 1e-3), k = 50:
    the BF16 margin band below the k-th score holds more candidates than the
    lists keep, so rows go to the rescan fallback; the hi/lo split proves a
    margin an order of magnitude tighter, and both stay exact."""
    nA, nB, d, k = 256, 20000, 256, 50
    C = datagen.centres(1, d, 73)
    A = datagen.clustered(nA, d, 1, 0.1, seed=73, stream=0, C=C)
    B = datagen.clustered(nB, d, 1, 0.1, seed=73, stream=1, C=C)
    out = {}
    for prec in ("bf16", "bf16x3"):
        J = sjmod.SimilarityJoin(d, prec=prec, device=0)
        idx, sc, st = J.topk(dev(A), dev(B), k, with_stats=True)
        J.close()
        assert_topk(idx, sc, A, B, k)
        assert st["max_abs_err_lowprec"] <= st["margin_max"]
        out[prec] = st
    assert out["bf16x3"]["margin_max"] < out["bf16"]["margin_max"] / 4
    assert out["bf16"]["n_overflow_rows"] > 0
    assert out["bf16x3"]["n_overflow_rows"] < out["bf16"]["n_overflow_rows"]
    assert out["bf16x3"]["n_rescored"] < out["bf16"]["n_rescored"]


def test_cascade_reaches_every_stage_on_massive_ties(sjmod):
    """200 one-hot rows over 2 keys against 1,300: every row has ~650 exact
    ties at its k-th score, more than any band list holds.  The BF16 pass
    overflows, the rows are re-joined in the hi/lo split (overflow again:
    the ties are exact), then in FP32 (again), and finally re-ranked against
    all of B by the rescan; the results stay exact throughout."""
    keys, k = 2, 10
    A = datagen.one_hot(datagen.keys(200, keys, 61, 0), keys)
    B = datagen.one_hot(datagen.keys(1300, keys, 61, 1), keys)
    J = sjmod.SimilarityJoin(keys, prec="bf16", device=0, flags=sjmod.SJ_FLAG_SINGLE_SPLIT)
    idx, sc, st = J.topk(dev(A), dev(B), k, with_stats=True)
    J.close()
    assert_topk(idx, sc, A, B, k)
    assert st["n_overflow_rows"] == 200
    assert st["n_rejoined_rows"] == 200 and st["n_rejoined_again"] == 200


@pytest.mark.parametrize("prec", ("fp8", "bf16"))
def test_cascade_dense_cluster_top50(sjmod, prec):
    """One dense cluster, k = 50, one column split per row block (each row's
    candidates in two lists, as in joins of many rows): the E4M3 (or BF16)
    margin band overflows the lists of every row; the re-join in the hi/lo
    split, with band lists sized by the columns they cover, settles almost
    all of them on the tensor cores."""
    nA, nB, d, k = 300, 20000, 256, 50
    C = datagen.centres(1, d, 74)
    A = datagen.clustered(nA, d, 1, 0.1, seed=74, stream=0, C=C)
    B = datagen.clustered(nB, d, 1, 0.1, seed=74, stream=1, C=C)
    J = sjmod.SimilarityJoin(d, prec=prec, device=0, flags=sjmod.SJ_FLAG_SINGLE_SPLIT)
    idx, sc, st = J.topk(dev(A), dev(B), k, with_stats=True)
    J.close()
    assert_topk(idx, sc, A, B, k)
    assert st["n_overflow_rows"] >= 64
    assert st["n_rejoined_rows"] == st["n_overflow_rows"]
    assert st["n_rejoined_again"] < st["n_rejoined_rows"] // 4
