"""The widest embeddings the library is built for (d = 16, 20, 25 and the
maximum, 32) through the whole nested loop against the FP64 oracle.

These d give row mappings the narrow cases do not: 25 columns leave one
row per warp with lanes idle (no vector loads), 20 and 32 put four FP32
columns on a lane, and the d x d Gram and polar factor reach their largest
size (528 Gram entries).  Ragged n, radius 2 and 3 graphs; tolerances as
in the other parity tests (FP64 <= 1e-9, mixed <= 2e-4) plus the
constraint Yhat^T D Yhat = I of Eq. 2."""
import numpy as np
import pytest

from oracle import pfe_oracle as O
from synth import make_problem
from tests.gpu_common import gpu_problem, oracle_graph, relerr, small_spec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-9), ("mixed", 1e-6, 2e-4)])
@pytest.mark.parametrize("d,radius", [(16, 2.0), (20, 3.0), (25, 2.0), (32, 3.0)])
def test_wide_embeddings_match_oracle(d, radius, precision, tol, bound):
    spec = small_spec(H=14, W=17, d=d, radius=radius)
    X, Y0 = make_problem(spec)
    g = oracle_graph(spec, X)
    ost = O.soc_pfe(g, Y0, 2, 3, solver="direct")
    p, _, _ = gpu_problem(spec, precision, tol=tol)
    p.init(Y0)
    Y = np.empty((spec.n, d))
    Yhat = np.empty((spec.n, d))
    p.solve(2, 3, Y, Yhat)
    assert relerr(Y, ost.Y) <= bound
    assert relerr(Yhat, O.embedding(g, ost)) <= bound
    assert np.max(np.abs(Yhat.T @ (g.dvec[:, None] * Yhat) - np.eye(d))) <= 1e-10
    p.close()


def test_dimension_beyond_the_maximum_is_rejected():
    from paper_1612_06496_gb300 import PFEError
    spec = small_spec(H=14, W=17, d=3)
    p, _, _ = gpu_problem(spec, "mixed")
    for d in (33, 17, 26):  # above the maximum, and two widths between the built ones
        with pytest.raises(PFEError) as ei:
            p.init(np.random.default_rng(d).standard_normal((spec.n, d)))
        assert ei.value.status == 8
    p.close()
