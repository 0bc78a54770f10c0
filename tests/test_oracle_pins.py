"""Pins for the oracle: checks against things other than the oracle itself.

* brute force with exact rational arithmetic (fractions.Fraction) on tiny
  inputs, including exact ties, ties below FP64 resolution and rounding
  midpoints;
* the paper's own construction (Sec. 3.1): with one-hot rows the threshold
  join at any tau in (0, 1] is the equi-join, which a dictionary computes;
* the multi-attribute generalisation of Sec. 3.1 and Hadamard closed forms;
* invariants: self-join symmetry, monotonicity in tau, top-k prefix property,
  each record its own top-1 in a self-join;
* InfoNCE closed forms and FP64 finite differences.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2112_07552_gb300 import datagen


# --------------------------------------------------------------------------
# independent exact helpers (Fraction based; nothing shared with the oracle)
# --------------------------------------------------------------------------

def fdot(a, b) -> Fraction:
    return sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)), Fraction(0))


def rn_binary(x: Fraction, p: int, qmin: int) -> Fraction:
    """Round-to-nearest-even to p significant bits, quantum >= 2^qmin."""
    if x == 0:
        return Fraction(0)
    sign = 1 if x > 0 else -1
    ax = abs(x)
    e = ax.numerator.bit_length() - ax.denominator.bit_length()
    while Fraction(2) ** e > ax:
        e -= 1
    while Fraction(2) ** (e + 1) <= ax:
        e += 1
    q = max(e - (p - 1), qmin)
    M = round(ax / Fraction(2) ** q)  # round() on a Fraction is half-to-even
    return sign * M * Fraction(2) ** q


def rn32(x: Fraction) -> np.float32:
    v = rn_binary(x, 24, -149)
    if abs(v) >= Fraction(2) ** 128:
        return np.float32(np.inf if v > 0 else -np.inf)
    return np.float32(float(v))


def brute_topk(A, B, k):
    out = []
    for a in A:
        s = [(fdot(a, b), j) for j, b in enumerate(B)]
        s.sort(key=lambda t: (-t[0], t[1]))
        out.append(s[:k])
    return out


def check_topk(A, B, k):
    idx, s32, s64 = oracle.topk(A, B, k)
    ref = brute_topk(A, B, k)
    for i, row in enumerate(ref):
        for r in range(k):
            if r < len(row):
                s, j = row[r]
                assert idx[i, r] == j, (i, r)
                assert s32[i, r] == rn32(s), (i, r)
                assert s64[i, r] == float(s), (i, r)
            else:
                assert idx[i, r] == -1 and s32[i, r] == -np.inf and s64[i, r] == -np.inf


def check_threshold(A, B, tau):
    i, j, s32, s64 = oracle.threshold(A, B, tau)
    exp = []
    for ii, a in enumerate(A):
        for jj, b in enumerate(B):
            s = fdot(a, b)
            if s >= Fraction(tau):
                exp.append((ii, jj, rn32(s), float(s)))
    assert len(exp) == len(i)
    for t, (ii, jj, e32, e64) in enumerate(exp):
        assert (i[t], j[t]) == (ii, jj)
        assert s32[t] == e32
        assert s64[t] == e64


def rand_floats(rng, shape, lo_exp=-30, hi_exp=2):
    m = rng.uniform(1.0, 2.0, size=shape)
    e = rng.integers(lo_exp, hi_exp, size=shape)
    s = rng.choice([-1.0, 1.0], size=shape)
    return (s * np.ldexp(m, e)).astype(np.float32)


# --------------------------------------------------------------------------
# exact accumulator and rounding
# --------------------------------------------------------------------------

def test_exact_dot_matches_fractions():
    rng = np.random.default_rng(1)
    for trial in range(300):
        d = int(rng.integers(1, 40))
        a = rand_floats(rng, d, -140, 60)
        b = rand_floats(rng, d, -140, 60)
        # sprinkle zeros and subnormals
        a[rng.random(d) < 0.1] = 0.0
        b[rng.random(d) < 0.05] = np.float32(1e-42)
        assert oracle.exact_dot(a, b) == fdot(a, b)


def test_exact_rounding_matches_fractions():
    rng = np.random.default_rng(2)
    for trial in range(400):
        d = int(rng.integers(1, 24))
        a = rand_floats(rng, d, -80, 3)
        b = rand_floats(rng, d, -80, 3)
        s32, s64 = oracle.exact_dot_rounded(a, b)
        x = fdot(a, b)
        assert s32 == rn32(x)
        assert s64 == float(x)


@pytest.mark.parametrize("a,b,want", [
    # 1 + 2^-24 is the midpoint of 1 and 1 + 2^-23: ties to even -> 1
    ([1.0, 2.0 ** -24], [1.0, 1.0], 1.0),
    # a hair above the midpoint (invisible to an FP64 naive sum) rounds up
    ([1.0, 2.0 ** -24, 2.0 ** -70], [1.0, 1.0, 1.0], 1.0 + 2.0 ** -23),
    # a hair below rounds down
    ([1.0, 2.0 ** -24, -(2.0 ** -70)], [1.0, 1.0, 1.0], 1.0),
    # midpoint above an odd mantissa rounds to the even neighbour above
    ([1.0 + 2.0 ** -23, 2.0 ** -24], [1.0, 1.0], 1.0 + 2.0 ** -22),
    # subnormal result
    ([2.0 ** -100], [2.0 ** -60], 0.0),
    ([2.0 ** -70], [2.0 ** -70], 2.0 ** -140),
])
def test_rounding_midpoints(a, b, want):
    a = np.array(a, np.float32)
    b = np.array(b, np.float32)
    s32, _ = oracle.exact_dot_rounded(a, b)
    assert s32 == np.float32(want)
    assert s32 == rn32(fdot(a, b))


# --------------------------------------------------------------------------
# brute force on tiny joins
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_topk_threshold_bruteforce_random(seed):
    rng = np.random.default_rng(100 + seed)
    nA, nB, d = int(rng.integers(1, 12)), int(rng.integers(1, 14)), int(rng.integers(1, 9))
    A = datagen.unit_rows(nA, d, seed, 0)
    B = datagen.unit_rows(nB, d, seed, 1)
    # exact duplicates and negations in B create exact ties
    if nB >= 3:
        B[1] = B[0]
        B[2] = -B[0]
    for k in (1, 3, nB, nB + 2):
        check_topk(A, B, k)
    for tau in (-1.5, -0.2, 0.0, 0.3, 0.9):
        check_threshold(A, B, tau)


def test_ties_below_fp64_resolution():
    # s_j = 1/2 + t_j 2^-80: an FP64 naive sum sees 1/2 for every j.
    rng = np.random.default_rng(7)
    t = rng.integers(-4, 5, size=25)
    A = np.array([[1.0, 2.0 ** -40]], np.float32)
    B = np.stack([np.full(25, 0.5), t * 2.0 ** -40], axis=1).astype(np.float32)
    idx, s32, _ = oracle.topk(A, B, 25)
    want = sorted(range(25), key=lambda j: (-t[j], j))
    assert list(idx[0]) == want
    assert np.all(s32 == np.float32(0.5))
    i, j, _, _ = oracle.threshold(A, B, 0.5)
    assert list(j) == [jj for jj in range(25) if t[jj] >= 0]
    check_topk(A, B, 7)


def test_fp64_sum_error_is_enclosed():
    # 1 + 1024 * 2^-53: every naive FP64 addition 1 + 2^-53 rounds back to 1,
    # so the FP64 sum is 1 while the exact value is 1 + 2^-43 -- an error of
    # 1024 ulps, which only the gamma_d * sum|p| term of the enclosure covers.
    # A second row scores exactly 1 + 2^-45 (above the naive sum, below the
    # exact value).
    d = 1025
    a = np.full(d, 2.0 ** -27, np.float32)
    a[0] = 1.0
    b0 = np.full(d, 2.0 ** -26, np.float32)
    b0[0] = 1.0
    b1 = np.zeros(d, np.float32)
    b1[0] = 1.0
    b1[1] = 2.0 ** -18
    A, B = a[None, :], np.stack([b1, b0])
    assert fdot(a, b0) == 1 + Fraction(2) ** -43
    assert fdot(a, b1) == 1 + Fraction(2) ** -45
    idx, _, s64 = oracle.topk(A, B, 1)
    assert idx[0, 0] == 1 and s64[0, 0] == 1 + 2.0 ** -43
    check_topk(A, B, 2)
    _, j, _, _ = oracle.threshold(A, B, 1 + 2.0 ** -44)
    assert list(j) == [1]


def test_threshold_is_inclusive():
    # <a, b> = 0.75 exactly: tau = 0.75 keeps the pair, the next double drops it.
    A = np.array([[0.5, 0.5]], np.float32)
    B = np.array([[1.0, 0.5], [1.0, 0.25]], np.float32)
    _, j, s32, _ = oracle.threshold(A, B, 0.75)
    assert list(j) == [0] and s32[0] == np.float32(0.75)
    _, j, _, _ = oracle.threshold(A, B, np.nextafter(0.75, 1.0))
    assert list(j) == []
    _, j, _, _ = oracle.threshold(A, B, 0.625)
    assert list(j) == [0, 1]


@pytest.mark.parametrize("tau", [2.0 ** -1074, -2.0 ** -1074, 2.0 ** -1068, -2.0 ** -1068,
                                 2.0 ** -1022, 2.0 ** -298, -2.0 ** -298, 0.0, -0.0])
def test_threshold_subnormal_tau(tau):
    # Every nonzero score is a multiple of 2^-298, so a tau between 0 and that
    # quantum separates the exactly-zero pairs from the tiny positive ones:
    # s = 0 is kept only for tau <= 0, s = 2^-298 for tau <= 2^-298.
    t = np.float32(2.0 ** -149)
    A = np.array([[1.0, 1.0, 0.0], [t, 0.0, 0.0]], np.float32)
    B = np.array([[1.0, -1.0, 0.0],     # s = 0 with row 0
                  [t, 0.0, 0.0],        # s = 2^-149 with row 0, 2^-298 with row 1
                  [-t, 0.0, 0.0],       # negatives of the above
                  [0.0, 0.0, 1.0]], np.float32)
    check_threshold(A, B, tau)
    _, j, _, _ = oracle.threshold(A[:1], B[:1], tau)
    assert list(j) == ([0] if tau <= 0 else [])
    # the exact difference s - tau every such decision takes the sign of
    for a in A:
        for b in B:
            assert oracle.exact_dot_minus(a, b, tau) == fdot(a, b) - Fraction(tau)


def test_exact_dot_minus_matches_fractions():
    # s - t exactly, for t over the whole double range (subnormal to 2^290)
    rng = np.random.default_rng(7)
    ts = [2.0 ** -1074, 3 * 2.0 ** -1074, 2.0 ** -1060 * 1.75, 2.0 ** -1022, 2.0 ** -700,
          0.85, 1.0 - 2.0 ** -53, 2.0 ** 100 * 1.5, 2.0 ** 290]
    for trial in range(200):
        d = int(rng.integers(1, 20))
        a = rand_floats(rng, d, -140, 4)
        b = rand_floats(rng, d, -140, 4)
        t = ts[trial % len(ts)] * (-1.0 if trial % 2 else 1.0)
        assert oracle.exact_dot_minus(a, b, t) == fdot(a, b) - Fraction(t), (trial, t)


# --------------------------------------------------------------------------
# the paper's construction: one-hot rows make the join an equi-join (Sec. 3.1)
# --------------------------------------------------------------------------

def hash_join(ka, kb):
    by_key = {}
    for j, v in enumerate(kb):
        by_key.setdefault(int(v), []).append(j)
    pairs = []
    for i, v in enumerate(ka):
        for j in by_key.get(int(v), []):
            pairs.append((i, j))
    return pairs


def _em_shapes():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "em_blocking_shapes.json")) as f:
        g = json.load(f)
    beer, itunes = g["beeradvo_ratebeer"], g["itunes_amazon"]
    return [
        # BeerAdvo-RateBeer tables joined on ABV (Sec. 6.3.2)
        (beer["rows"][0], beer["rows"][1], beer["distinct"]["ABV"]),
        # a 10% slice of iTunes-Amazon joined on Price
        (itunes["rows"][0] // 10, itunes["rows"][1] // 10, itunes["distinct"]["Price"]),
    ]


@pytest.mark.parametrize("nA,nB,distinct", _em_shapes())
def test_one_hot_threshold_is_equi_join(nA, nB, distinct):
    ka = datagen.keys(nA, distinct, 0, 0)
    kb = datagen.keys(nB, distinct, 0, 1)
    A = datagen.one_hot(ka, distinct)
    B = datagen.one_hot(kb, distinct)
    want = hash_join(ka, kb)
    for tau in (2.0 ** -30, 0.5, 1.0):
        i, j, s32, _ = oracle.threshold(A, B, tau, want_s64=False)
        got = list(zip(i.tolist(), j.tolist()))
        assert got == want
        assert np.all(s32 == 1.0)
    i, _, _, _ = oracle.threshold(A, B, 1.0 + 2.0 ** -20, want_s64=False)
    assert len(i) == 0


def test_one_hot_topk_lowest_index_matches():
    nA, nB, distinct, k = 300, 500, 40, 10
    ka = datagen.keys(nA, distinct, 1, 0)
    kb = datagen.keys(nB, distinct, 1, 1)
    A, B = datagen.one_hot(ka, distinct), datagen.one_hot(kb, distinct)
    idx, s32, _ = oracle.topk(A, B, k)
    for i in range(nA):
        match = [j for j in range(nB) if kb[j] == ka[i]]
        rest = [j for j in range(nB) if kb[j] != ka[i]]
        want = (match + rest)[:k]
        assert list(idx[i]) == want
        assert list(s32[i]) == [1.0] * min(k, len(match)) + [0.0] * (k - min(k, len(match)))


def test_multi_attribute_one_hot_counts_matches():
    # Sec. 3.1: ID/Val generalise to attribute sets; with 4 attributes scaled by
    # 1/2 the score is exactly (#equal attributes)/4.
    doms = (5, 7, 11, 13)
    nA, nB = 150, 120
    ka = [datagen.keys(nA, v, 3, s) for s, v in enumerate(doms)]
    kb = [datagen.keys(nB, v, 3, 10 + s) for s, v in enumerate(doms)]
    A = datagen.multi_attr_one_hot(ka, doms)
    B = datagen.multi_attr_one_hot(kb, doms)
    cnt = sum((ka[t][:, None] == kb[t][None, :]).astype(int) for t in range(4))
    for tau in (0.25, 0.5, 1.0):
        i, j, s32, _ = oracle.threshold(A, B, tau, want_s64=False)
        wi, wj = np.nonzero(cnt >= 4 * tau)
        assert np.array_equal(i, wi) and np.array_equal(j, wj)
        assert np.array_equal(s32, (cnt[wi, wj] / 4.0).astype(np.float32))
    idx, s32, _ = oracle.topk(A, B, 6)
    for r in range(nA):
        want = sorted(range(nB), key=lambda jj: (-cnt[r, jj], jj))[:6]
        assert list(idx[r]) == want


def sylvester(n):
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H


def test_hadamard_closed_form():
    H = (sylvester(256) / 16.0).astype(np.float32)   # orthonormal rows
    A = H[:64]
    B = np.concatenate([H[32:96], -H[:16]], axis=0)  # 80 rows
    idx, s32, _ = oracle.topk(A, B, 3)
    for i in range(64):
        if i >= 32:
            # B[i-32] == H[i]: score 1, then zeros in index order
            want = [i - 32] + [j for j in range(80) if j != i - 32][:2]
            assert list(s32[i]) == [1.0, 0.0, 0.0]
        else:
            want = [j for j in range(80) if not (j == 64 + i)][:3]
            assert list(s32[i]) == [0.0, 0.0, 0.0]
        assert list(idx[i]) == want
    i, j, s32, _ = oracle.threshold(A, B, -1.0)
    assert len(i) == 64 * 80
    S = (A.astype(np.float64) @ B.astype(np.float64).T)
    assert np.array_equal(s32.reshape(64, 80), S.astype(np.float32))


# --------------------------------------------------------------------------
# invariants on clustered data
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def clustered_small():
    return datagen.clustered(240, 24, 12, sigma=0.3, seed=5)


def test_self_join_symmetry(clustered_small):
    X = clustered_small
    n = X.shape[0]
    i, j, s32, s64 = oracle.threshold(X, X, -2.0)
    assert len(i) == n * n
    S32 = s32.reshape(n, n)
    S64 = s64.reshape(n, n)
    assert np.array_equal(S32, S32.T)
    assert np.array_equal(S64, S64.T)


def test_monotone_in_tau(clustered_small):
    X = clustered_small
    prev = None
    for tau in (0.2, 0.5, 0.8, 0.95, 0.99):
        i, j, _, _ = oracle.threshold(X, X, tau, want_s64=False)
        cur = set(zip(i.tolist(), j.tolist()))
        if prev is not None:
            assert cur <= prev
        prev = cur


def test_topk_prefix_and_own_top1(clustered_small):
    X = clustered_small
    i5, s5, _ = oracle.topk(X, X, 5)
    i12, s12, _ = oracle.topk(X, X, 12)
    assert np.array_equal(i5, i12[:, :5]) and np.array_equal(s5, s12[:, :5])
    i1, _, _ = oracle.topk(X, X, 1)
    for r in range(X.shape[0]):
        j = i1[r, 0]
        assert j == r or (j < r and oracle.exact_dot(X[r], X[j]) == oracle.exact_dot(X[r], X[r]))


def test_threshold_equals_filtered_full_ranking(clustered_small):
    X = clustered_small
    n = X.shape[0]
    idx, s32, s64 = oracle.topk(X, X, n)
    tau = 0.7
    i, j, t32, _ = oracle.threshold(X, X, tau, want_s64=False)
    for r in range(n):
        sel = [jj for jj, v in zip(idx[r], s64[r]) if oracle.exact_dot(X[r], X[jj]) >= Fraction(tau)]
        got = j[i == r].tolist()
        assert sorted(sel) == got


def test_sampled_rows_match_full(clustered_small):
    X = clustered_small
    rows = np.array([5, 0, 239, 17])
    idx, s32, _ = oracle.topk(X, X, 7)
    ridx, rs32, _ = oracle.topk(X, X, 7, rows=rows)
    assert np.array_equal(ridx, idx[rows]) and np.array_equal(rs32, s32[rows])


def test_empty_inputs():
    A = np.zeros((0, 8), np.float32)
    B = datagen.unit_rows(5, 8, 0, 0)
    idx, _, _ = oracle.topk(A, B, 3)
    assert idx.shape == (0, 3)
    idx, s32, _ = oracle.topk(B, np.zeros((0, 8), np.float32), 3)
    assert np.all(idx == -1) and np.all(s32 == -np.inf)
    i, j, _, _ = oracle.threshold(B, np.zeros((0, 8), np.float32), 0.0)
    assert len(i) == 0


# --------------------------------------------------------------------------
# InfoNCE
# --------------------------------------------------------------------------

def test_infonce_identical_rows():
    N, d, T = 17, 6, 0.05
    a = datagen.unit_rows(1, d, 0, 0)[0]
    b = datagen.unit_rows(1, d, 0, 1)[0]
    A = np.tile(a.astype(np.float64), (N, 1))
    B = np.tile(b.astype(np.float64), (N, 1))
    loss, lse, _, dA, dB = oracle.infonce(A, B, T)
    assert loss == pytest.approx(np.log(N), rel=1e-13)
    assert np.max(np.abs(dA)) < 1e-12 and np.max(np.abs(dB)) < 1e-12


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("T,rtol", [(0.5, 1e-12), (0.05, 1e-6)])
def test_infonce_identity_closed_form(sym, T, rtol):
    # A = B = I_N: S = I/T, l_i = log(e^{1/T} + N - 1), L = l - 1/T.
    # (At T = 0.05 the oracle's P_ii - 1 cancels: e^20/Z - 1 loses ~8 digits.)
    N = 12
    I = np.eye(N)
    loss, lse, lse_c, dA, dB = oracle.infonce(I, I, T, sym=sym)
    Z = np.exp(1.0 / T) + N - 1
    assert loss == pytest.approx(np.log(Z) - 1.0 / T, rel=1e-12)
    G = np.full((N, N), 1.0 / Z)
    np.fill_diagonal(G, -(N - 1) / Z)   # P_ii - 1 without cancellation
    G /= N
    # identity inputs: dA[i, :] = sum_j G_ij e_j / T = G[i, :] / T
    assert np.allclose(dA, G / T, rtol=rtol, atol=0)
    assert np.allclose(dB, G.T / T, rtol=rtol, atol=0)


@pytest.mark.parametrize("sym", [False, True])
def test_infonce_finite_differences(sym):
    # 64 x 64 pairs, d = 32: FP64 central differences of the oracle loss.
    N, d, T = 64, 32, 0.05
    A, B = datagen.paired(N, d, 8, seed=11)
    A = A.astype(np.float64)
    B = B.astype(np.float64)
    g = 0.7
    loss, _, _, dA, dB = oracle.infonce(A, B, T, sym=sym, g=g)
    rng = np.random.default_rng(3)
    h = 1e-6
    for X, dX in ((A, dA), (B, dB)):
        for _ in range(40):
            i, k = int(rng.integers(N)), int(rng.integers(d))
            old = X[i, k]
            X[i, k] = old + h
            lp = oracle.infonce(A, B, T, sym=sym, grads=False)[0]
            X[i, k] = old - h
            lm = oracle.infonce(A, B, T, sym=sym, grads=False)[0]
            X[i, k] = old
            fd = g * (lp - lm) / (2 * h)
            assert abs(fd - dX[i, k]) <= 1e-7 * max(1.0, abs(dX[i, k])) + 1e-9


def test_infonce_rows_match_full():
    N, d, T = 40, 16, 0.1
    A, B = datagen.paired(N, d, 4, seed=12)
    loss, lse, _, dA, _ = oracle.infonce(A, B, T, g=1.3)
    rows = np.array([0, 7, 39])
    l2, dA2 = oracle.infonce_rows(A, B, T, rows, g=1.3)
    assert np.allclose(l2, lse[rows], rtol=1e-14)
    assert np.allclose(dA2, dA[rows], rtol=1e-12, atol=1e-15)


def test_enclose_all_contains_the_exact_score():
    # the FP64 enclosure used for the every-pair margin check: lo <= s <= hi
    # for the exact s (Fraction), and it is tight (width far below 1e-12 here)
    rng = np.random.default_rng(11)
    A = rand_floats(rng, (12, 37), -20, 1)
    B = rand_floats(rng, (9, 37), -20, 1)
    lo, hi = oracle.enclose_all(A, B)
    for i in range(A.shape[0]):
        for j in range(B.shape[0]):
            s = fdot(A[i], B[j])
            assert Fraction(lo[i, j]) <= s <= Fraction(hi[i, j]), (i, j)
            assert hi[i, j] - lo[i, j] <= 1e-12 * max(1.0, abs(float(s)))
