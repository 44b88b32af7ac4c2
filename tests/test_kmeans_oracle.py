"""Pins of the k-means oracle (segmentation stage of Sec. IV): a library
Lloyd implementation from the same start, separated clusters, fixed point
and monotone objective."""
import numpy as np
import pytest

from oracle import kmeans_oracle as K


def _blobs(seed=0, k=4, per=50, d=3, spread=0.05):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-1, 1, size=(k, d)) * 4
    X = np.vstack([c + spread * rng.standard_normal((per, d)) for c in centers])
    truth = np.repeat(np.arange(k), per)
    perm = rng.permutation(X.shape[0])
    return X[perm], truth[perm]


def test_separated_blobs_recovered():
    X, truth = _blobs()
    labels, C, inertia, rounds = K.kmeans(X, 4)
    # the same partition up to a relabelling
    pairs = {(int(a), int(b)) for a, b in zip(labels, truth)}
    assert len(pairs) == 4 and len({a for a, _ in pairs}) == 4


def test_matches_library_lloyd_from_the_same_start():
    sk = pytest.importorskip("sklearn.cluster")
    X, _ = _blobs(seed=3, k=5, per=40, d=4, spread=0.6)
    C0 = K.maximin_init(X, 5)
    labels, C, inertia, _ = K.lloyd(X, C0, 300)
    ref = sk.KMeans(n_clusters=5, init=C0, n_init=1, algorithm="lloyd", max_iter=300, tol=0.0).fit(X)
    np.testing.assert_array_equal(labels, ref.labels_)
    np.testing.assert_allclose(C, ref.cluster_centers_, atol=1e-10)
    assert abs(inertia - ref.inertia_) <= 1e-9 * ref.inertia_


def test_fixed_point_and_monotone_inertia():
    X, _ = _blobs(seed=5, k=6, per=30, d=3, spread=0.8)
    C = K.maximin_init(X, 6)
    prev = np.inf
    for _ in range(20):  # one Lloyd round at a time: the objective never increases
        labels, C, inertia, _ = K.lloyd(X, C, 1)
        assert inertia <= prev + 1e-12
        prev = inertia
    labels, C, inertia, _ = K.lloyd(X, C, 500)
    D = K.sq_dist(X, C)
    np.testing.assert_array_equal(labels, np.argmin(D, axis=1))          # nearest centroid
    for j in range(6):
        np.testing.assert_allclose(C[j], X[labels == j].mean(axis=0))    # means of their rows


def test_maximin_start_by_hand():
    X = np.array([[0.0, 0.0], [1.0, 0.0], [5.0, 0.0], [5.0, 1.0], [-3.0, 0.0]])
    C = K.maximin_init(X, 3)
    np.testing.assert_array_equal(C[0], X[0])
    np.testing.assert_array_equal(C[1], X[3])   # farthest from row 0: |(5, 1)|^2 = 26
    np.testing.assert_array_equal(C[2], X[4])   # then min distances: 1, 1, 0, 0, 9 -> row 4
