"""Pins for the relational oracle (oracle/relational.py), against things
other than itself: brute-force pair enumeration with exact arithmetic, the
dictionary hash join, the similarity-join oracle on the paper's one-hot
encoding (Sec. 3.1: C = mat(A) mat(B)^T), and the paper's matrix formulas
for Q3 (1 x mat(A) x mat(B)^T) and Q4 (sum of mat(A) mat(B)^T) in exact
integer arithmetic (Sec. 3.3)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import relational
from paper_2112_07552_gb300 import datagen
from test_oracle_pins import hash_join, rn32


def brute_block(ka, kb, m):
    n = ka.shape[1]
    c = Fraction(float(np.float32(1.0 / np.sqrt(n))))
    out = []
    for i in range(ka.shape[0]):
        for j in range(kb.shape[0]):
            eq = int(np.sum(ka[i] == kb[j]))
            if eq >= m:
                out.append((i, j, rn32(eq * c * c)))
    return out


@pytest.mark.parametrize("n_attr", [1, 2, 3, 4])
def test_block_matches_brute_force(n_attr):
    rng = np.random.default_rng(n_attr)
    ka = rng.integers(0, 4, size=(37, n_attr))
    kb = rng.integers(0, 4, size=(29, n_attr))
    for m in range(1, n_attr + 1):
        i, j, s = relational.block(ka, kb, m)
        want = brute_block(ka, kb, m)
        assert [(a, b) for a, b, _ in want] == list(zip(i.tolist(), j.tolist()))
        assert np.array_equal(np.array([x for _, _, x in want], np.float32).view(np.uint32),
                              s.view(np.uint32))


def test_block_single_attribute_is_the_hash_join():
    ka = datagen.keys(500, 12, 0, 0)
    kb = datagen.keys(700, 12, 0, 1)
    i, j, s = relational.block(ka, kb, 1)
    assert list(zip(i.tolist(), j.tolist())) == sorted(hash_join(ka, kb))
    assert np.all(s == 1.0)


def test_block_is_the_one_hot_product():
    # the paper's construction: one-hot blocks per attribute, C = A B^T; the
    # pairs with >= m equal attributes are those with C_ij >= (m - 1/2) / n
    rng = np.random.default_rng(9)
    doms = [5, 3, 7, 4]
    ka = np.stack([rng.integers(0, v, size=60) for v in doms], axis=1)
    kb = np.stack([rng.integers(0, v, size=45) for v in doms], axis=1)
    A = datagen.multi_attr_one_hot(ka.T, doms)
    B = datagen.multi_attr_one_hot(kb.T, doms)
    for m in range(1, 5):
        i, j, s = relational.block(ka, kb, m)
        wi, wj, ws, _ = oracle.threshold(A, B, (m - 0.5) / 4)
        assert np.array_equal(i, wi) and np.array_equal(j, wj)
        assert np.array_equal(s.view(np.uint32), ws.view(np.uint32))
        assert np.all(s * 4 == np.round(s * 4))  # scale 1/2: scores are matches / 4


def brute_q3(a_id, a_val, b_id, b_g):
    acc = {}
    for ia, va in zip(a_id.tolist(), a_val.tolist()):
        for ib, gb in zip(b_id.tolist(), b_g.tolist()):
            if ia == ib:
                s, c = acc.get(gb, (0, 0))
                acc[gb] = (s + va, c + 1)
    return [(g, s, c) for g, (s, c) in sorted(acc.items())]


def brute_q4(a_id, a_val, b_id, b_val):
    tot = cnt = 0
    for ia, va in zip(a_id.tolist(), a_val.tolist()):
        for ib, vb in zip(b_id.tolist(), b_val.tolist()):
            if ia == ib:
                tot += va * vb
                cnt += 1
    return tot, cnt


def test_groupby_and_sum_product_match_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(20):
        nA, nB = int(rng.integers(0, 40)), int(rng.integers(0, 40))
        a_id = rng.integers(-3, 8, size=nA)
        b_id = rng.integers(0, 10, size=nB)  # some keys of one side only
        a_val = rng.integers(-2 ** 31, 2 ** 31, size=nA)
        b_g = rng.integers(-5, 5, size=nB)
        b_val = rng.integers(-2 ** 31, 2 ** 31, size=nB)
        assert relational.groupby_sum(a_id, a_val, b_id, b_g) == brute_q3(a_id, a_val, b_id, b_g)
        assert relational.sum_product(a_id, a_val, b_id, b_val) == brute_q4(a_id, a_val, b_id, b_val)


def test_q3_q4_match_the_papers_matrix_formulas():
    # Q3 = 1 x mat(A) x mat(B)^T with mat(A)_iv = a_i.Val [a_i.ID = v] and the
    # 0/1 mat(B)_uv = [(u, v) in B]; Q4 = 1 x mat(A) mat(B)^T x 1 with
    # mat(B)_jv = b_j.Val [b_j.ID = v].  Exact integer matrices (object dtype).
    rng = np.random.default_rng(4)
    K, nA, nB = 6, 50, 40
    a_id = rng.integers(0, K, size=nA)
    a_val = rng.integers(-1000, 1000, size=nA)
    # B without duplicate (ID, G) tuples, so the 0/1 matrix of the paper applies
    pairs = sorted({(int(i), int(g)) for i, g in zip(rng.integers(0, K, size=nB),
                                                      rng.integers(0, 7, size=nB))})
    b_id = np.array([p[0] for p in pairs])
    b_g = np.array([p[1] for p in pairs])
    groups = sorted(set(b_g.tolist()))
    matA = np.zeros((nA, K), dtype=object)
    for i in range(nA):
        matA[i, a_id[i]] = int(a_val[i])
    matB = np.zeros((len(groups), K), dtype=object)
    for i, g in zip(b_id, b_g):
        matB[groups.index(int(g)), i] = 1
    M = np.ones((1, nA), dtype=object).dot(matA).dot(matB.T)[0]
    got = {g: s for g, s, _ in relational.groupby_sum(a_id, a_val, b_id, b_g)}
    for u, g in enumerate(groups):
        assert got.get(g, 0) == M[u]
    b_val = rng.integers(-1000, 1000, size=len(b_id))
    matB4 = np.zeros((len(b_id), K), dtype=object)
    for j in range(len(b_id)):
        matB4[j, b_id[j]] = int(b_val[j])
    q4 = np.ones((1, nA), dtype=object).dot(matA).dot(matB4.T).dot(
        np.ones((len(b_id), 1), dtype=object))[0, 0]
    assert relational.sum_product(a_id, a_val, b_id, b_val)[0] == q4
