"""k-means segmentation (Sec. IV) on the GPU against the oracle: seeded
points given to both, and the embedding each side computes itself."""
import numpy as np
import pytest

from oracle import kmeans_oracle as K
from oracle import pfe_oracle as O
from synth import CONFIGS, crop_specs
from tests.gpu_common import gpu_problem, oracle_graph, small_spec

pytestmark = pytest.mark.gpu


def _blobs(n, d, k, seed, spread):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-1, 1, size=(k, d)) * 3
    X = centers[rng.integers(0, k, n)] + spread * rng.standard_normal((n, d))
    return np.ascontiguousarray(X)


@pytest.mark.parametrize("start", ["maximin", "given"])
def test_kmeans_matches_oracle_on_points(start):
    spec = small_spec(H=50, W=100, d=3)  # any context of n = 5000 rows
    p, _, _ = gpu_problem(spec, "fp64")
    X = _blobs(spec.n, 5, 6, 11, 0.9)
    C0 = None if start == "maximin" else np.ascontiguousarray(X[[3, 70, 500, 1200, 2222, 4000]])
    labels, cent, inertia, rounds = p.kmeans(6, X=X, C0=C0, max_iter=200)
    ol, oc, oi, orr = K.lloyd(X, K.maximin_init(X, 6) if C0 is None else C0, 200)
    assert rounds == orr
    np.testing.assert_array_equal(labels, ol)
    np.testing.assert_allclose(cent, oc, rtol=0, atol=1e-12)
    assert abs(inertia - oi) <= 1e-12 * oi
    p.close()


def test_segmentation_of_the_embedding():
    """The segmentation of a 64x64 window of the benchmark image: k-means on
    each side's own FP64 embedding gives the same partition."""
    spec = crop_specs(CONFIGS["C5"])[0]
    p, X, Y0 = gpu_problem(spec, "fp64", tol=1e-12)
    g = oracle_graph(spec, X)
    p.init(Y0)
    p.solve(2, 5)
    labels, cent, inertia, rounds = p.kmeans(4)
    st = O.soc_pfe(g, Y0, 2, 5)
    ol, oc, oi, orr = K.kmeans(O.embedding(g, st), 4)
    np.testing.assert_array_equal(labels, ol)
    assert abs(inertia - oi) <= 1e-8 * max(oi, 1e-300)
    p.close()


def test_kmeans_argument_errors():
    from paper_1612_06496_gb300 import PFEError
    spec = small_spec(H=10, W=12, d=3)
    p, X, Y0 = gpu_problem(spec, "fp64")
    with pytest.raises(PFEError) as ei:
        p.kmeans(3)  # the embedding before pfe_init
    assert ei.value.status == 9
    with pytest.raises(PFEError) as ei:
        p.kmeans(65, X=np.zeros((spec.n, 2)))
    assert ei.value.status == 1
    p.close()
