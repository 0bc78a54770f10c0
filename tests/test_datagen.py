"""The seeded input generators: the recipe's claims that tests and the bench
rely on (determinism, independence from the thread count, unit rows, the
cluster and near-duplicate structure)."""
import numpy as np

from paper_2112_07552_gb300 import datagen


def test_same_data_for_any_thread_count(monkeypatch):
    a = datagen.clustered(20000, 64, 50, 0.1, seed=3, stream=0)
    monkeypatch.setattr(datagen, "_threads", lambda: 1)
    b = datagen.clustered(20000, 64, 50, 0.1, seed=3, stream=0)
    assert np.array_equal(a, b)


def test_streams_and_seeds_differ_and_rows_are_unit():
    a = datagen.clustered(3000, 96, 30, 0.1, seed=4, stream=0)
    b = datagen.clustered(3000, 96, 30, 0.1, seed=4, stream=1)
    c = datagen.clustered(3000, 96, 30, 0.1, seed=5, stream=0)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    for x in (a, b, c):
        n2 = np.einsum("ij,ij->i", x.astype(np.float64), x.astype(np.float64))
        assert np.all(np.abs(n2 - 1.0) <= 1e-6)


def test_total_noise_gives_within_cluster_cosine_near_0_99():
    # sigma is the total noise norm: members of one centre sit near cosine
    # 1 - sigma^2 = 0.99 of each other, different centres near 0
    C = datagen.centres(2, 256, 6)
    a = datagen.clustered(400, 256, 2, 0.1, seed=6, stream=0, C=C)
    asg = datagen.assignments(400, 2, 6, 0)
    S = a.astype(np.float64) @ a.astype(np.float64).T
    same = asg[:, None] == asg[None, :]
    np.fill_diagonal(same, False)
    diff = asg[:, None] != asg[None, :]
    assert abs(S[same].mean() - 0.99) < 0.003
    assert abs(S[diff].mean()) < 0.1


def test_zipf_assignment_is_heavy_headed():
    asg = datagen.assignments(200000, 50000, 0, 0, zipf_s=1.1)
    counts = np.bincount(asg, minlength=50000)
    top = np.sort(counts)[::-1]
    # Zipf(1.1) over 50,000 ranks: the largest cluster holds ~1/H(1.1) of the
    # rows (H = sum r^-1.1 ~ 9.6), the smallest ranks almost none
    H = np.sum(np.arange(1, 50001, dtype=np.float64) ** -1.1)
    assert abs(top[0] / 200000 - 1.0 / H) < 0.01
    assert np.count_nonzero(counts) < 50000


def test_near_duplicates_are_close_pairs():
    A = datagen.clustered(2000, 64, 200, 0.1, seed=7, stream=0)
    B = datagen.clustered(2000, 64, 200, 0.1, seed=7, stream=1)
    pairs = datagen.add_near_duplicates(A, B, 0.05, 0.02, seed=7)
    i, j = pairs[:, 0], pairs[:, 1]
    assert len(i) == 100
    cos = np.einsum("ij,ij->i", A[i].astype(np.float64), B[j].astype(np.float64))
    assert np.all(cos > 0.99)
