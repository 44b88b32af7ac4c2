"""Pins of the IC(0) oracle: the exact Cholesky factor where the pattern
holds it, (L L^T)_ij = A_ij on the pattern of A (the definition, checked by
a sparse product), positive pivots on the system matrix, and PCG with it."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import ic_oracle as I
from oracle import pfe_oracle as O
from synth import ImageSpec, make_problem


def _graph(H, W, radius, seed=4):
    spec = ImageSpec("t", H, W, 3, 0.05, seed=seed, radius=radius, sigma=0.1, d=2)
    X, _ = make_problem(spec)
    return O.build_grid_graph(X, H, W, radius, 0.1)


def test_ic0_is_the_cholesky_factor_of_a_tridiagonal_matrix():
    rng = np.random.default_rng(2)
    n = 40
    off = -rng.uniform(0.1, 1.0, n - 1)
    diag = np.abs(np.r_[off, 0.0]) + np.abs(np.r_[0.0, off]) + rng.uniform(0.1, 1.0, n)
    A = sp.diags([off, diag, off], [-1, 0, 1], format="csr")
    L = I.ic0(A)
    np.testing.assert_allclose(L.toarray(), sla.cholesky(A.toarray(), lower=True), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("radius", [2.0, 3.0])
def test_ic0_matches_a_on_its_pattern(radius):
    g = _graph(9, 11, radius)
    A = g.A.tocsr()
    L = I.ic0(A)
    assert np.all(L.diagonal() > 0)
    # the pattern of L is that of tril(A)
    pat = sp.tril(A).tocsr()
    pat.data[:] = 1.0
    lp = L.copy()
    lp.data[:] = 1.0
    assert (lp != pat).nnz == 0
    LLt = (L @ L.T).tocsr()
    P = A.copy()
    P.data[:] = 1.0
    on_pattern = LLt.multiply(P)
    np.testing.assert_allclose(on_pattern.toarray(), A.toarray(), rtol=1e-12, atol=1e-12 * abs(A).max())
    # and it is not the exact factor: fill-in is dropped
    assert abs((LLt - A)).max() > 1e-8 * abs(A).max()


def test_pcg_with_ic0_solves_and_beats_jacobi():
    g = _graph(20, 18, 2.0)
    L = I.ic0(g.A)
    Bm = np.random.default_rng(5).standard_normal((g.n, 3))
    X, info = O.pcg(g.A, Bm, np.zeros_like(Bm), 1e-10, 2000, 50, lambda R: I.ic0_apply(L, R))
    _, ij = O.jacobi_pcg(g.A, Bm, np.zeros_like(Bm), 1e-10, 2000)
    assert info["converged"] and info["iters"].max() < ij["iters"].max()
    np.testing.assert_allclose(X, O.DirectSolver(g.A)(Bm)[0], rtol=1e-7, atol=1e-9)
