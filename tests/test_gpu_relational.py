"""GPU parity of the relational patterns (sj_block, sj_join_groupby_sum,
sj_join_sum_product) against the relational oracle, at the paper's
entity-matching table shapes (Sec. 6.3.2: BeerAdvo-RateBeer 3,777 x 2,671,
iTunes-Amazon 6,907 x 55,923 with their printed distinct-value counts) and
at its microbenchmark shape (tables of (ID, Val) with 32 distinct IDs).
Pairs, their order and their float32 scores must be identical; aggregate
sums and counts are exact integers and must be equal."""
import json
import os

import numpy as np
import pytest

from oracle import relational
from paper_2112_07552_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "em_blocking_shapes.json")


@pytest.fixture(scope="module")
def J():
    from paper_2112_07552_gb300 import _build, sj
    _build.build()
    h = sj.SimilarityJoin(8, prec="bf16", device=0)
    yield h
    h.close()


def em_keys(name, attrs, side, seed=0):
    g = json.load(open(GOLD))[name]
    n = g["rows"][side]
    return np.stack([datagen.keys(n, g["distinct"][a], seed + t, side)
                     for t, a in enumerate(attrs)], axis=1)


def check_block(J, ka, kb, m, on_device=True):
    dev = (lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()) if on_device else \
        (lambda x: torch.from_numpy(np.ascontiguousarray(x)))
    i, j, s = J.block(dev(ka), dev(kb), m)
    wi, wj, ws = relational.block(ka, kb, m)
    assert np.array_equal(i.cpu().numpy(), wi) and np.array_equal(j.cpu().numpy(), wj)
    assert np.array_equal(s.cpu().numpy().view(np.uint32), ws.view(np.uint32))
    return len(wi)


def test_block_beer_abv_is_the_equi_join(J):
    ka = em_keys("beeradvo_ratebeer", ["ABV"], 0)
    kb = em_keys("beeradvo_ratebeer", ["ABV"], 1)
    assert check_block(J, ka, kb, 1) > 0


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_block_beer_four_attributes_m_of_4(J, m):
    attrs = ["ABV", "Style", "Factory", "BeerName"]
    ka = em_keys("beeradvo_ratebeer", attrs, 0)
    kb = em_keys("beeradvo_ratebeer", attrs, 1)
    check_block(J, ka, kb, m, on_device=(m % 2 == 0))


def test_block_itunes_price_32M_pairs(J):
    ka = em_keys("itunes_amazon", ["Price"], 0)
    kb = em_keys("itunes_amazon", ["Price"], 1)
    assert check_block(J, ka, kb, 1) > 30_000_000


@pytest.mark.parametrize("m", [1, 3, 6])
def test_block_itunes_six_attributes(J, m):
    attrs = ["Price", "Genre", "Time", "Artist", "Copyright", "Album"]
    ka = em_keys("itunes_amazon", attrs, 0)[:1500]
    kb = em_keys("itunes_amazon", attrs, 1)[:9000]
    check_block(J, ka, kb, m)


def test_block_edge_cases(J):
    # keys on one side only, negative and huge key values, empty sides
    ka = np.array([[-(2 ** 62)], [5], [7], [2 ** 62]], np.int64)
    kb = np.array([[5], [2 ** 62], [9], [5]], np.int64)
    assert check_block(J, ka, kb, 1) == 3
    assert check_block(J, ka[:0], kb, 1) == 0
    assert check_block(J, ka, kb[:0], 1) == 0


def tables(nA, nB, n_ids, n_groups, seed):
    rng = np.random.default_rng(seed)
    a_id = rng.integers(0, n_ids, size=nA).astype(np.int64)
    b_id = rng.integers(0, n_ids + n_ids // 4 + 1, size=nB).astype(np.int64)  # some miss
    a_val = rng.integers(-2 ** 31, 2 ** 31, size=nA).astype(np.int32)
    b_val = rng.integers(-2 ** 31, 2 ** 31, size=nB).astype(np.int32)
    b_g = rng.integers(-n_groups, n_groups, size=nB).astype(np.int64)
    return a_id, a_val, b_id, b_val, b_g


@pytest.mark.parametrize("nA,nB,n_ids,n_groups", [
    (32768, 32768, 32, 100),          # the paper's microbenchmark shape (32 distinct IDs)
    (300_000, 500_000, 5000, 3000),   # keys beyond the shared-memory privatisation
    (1, 1000, 1, 2000),
])
def test_groupby_and_sum_product(J, nA, nB, n_ids, n_groups):
    a_id, a_val, b_id, b_val, b_g = tables(nA, nB, n_ids, n_groups, nA + nB)
    dev = lambda x: torch.from_numpy(x).cuda()
    got = J.groupby_sum(dev(a_id), dev(a_val), dev(b_id), dev(b_g))
    assert got == relational.groupby_sum(a_id, a_val, b_id, b_g)
    assert J.sum_product(a_id, a_val, b_id, b_val) == \
        relational.sum_product(a_id, a_val, b_id, b_val)  # host inputs


def test_aggregates_extremes_and_empty(J):
    # every value at the int32 extremes on one key: sums far beyond 64 bits
    n = 200_000
    a_id = np.zeros(n, np.int64)
    a_val = np.full(n, -2 ** 31, np.int32)
    b_id = np.zeros(n, np.int64)
    b_val = np.full(n, -2 ** 31, np.int32)
    b_g = np.zeros(n, np.int64)
    got = J.groupby_sum(a_id, a_val, b_id, b_g)
    assert got == [(0, n * n * -2 ** 31, n * n)]
    assert J.sum_product(a_id, a_val, b_id, b_val) == (n * n * 2 ** 62, n * n)
    # no key in common, empty sides
    assert J.groupby_sum(a_id, a_val, b_id + 1, b_g) == []
    assert J.sum_product(a_id, a_val, b_id + 1, b_val) == (0, 0)
    assert J.groupby_sum(a_id[:0], a_val[:0], b_id, b_g) == []
    assert J.sum_product(a_id, a_val, b_id[:0], b_val[:0]) == (0, 0)
