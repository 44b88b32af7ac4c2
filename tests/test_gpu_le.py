"""GPU Laplacian-eigenmap start against the oracle's (dense / shift-invert
eigensolvers): vectors, sign rule, closed forms, null spaces, invariants."""
import numpy as np
import pytest

from oracle import pfe_oracle as O
from synth import CONFIGS
from tests.gpu_common import ensure_built, gpu_problem, oracle_graph, relerr

pytestmark = pytest.mark.gpu


def _align(V, E):
    """Columns of V against E: the sign rule decides, except where the two
    largest magnitudes of E's column tie to 1e-6 (rounding then picks it)."""
    out = V.copy()
    for c in range(E.shape[1]):
        a = np.sort(np.abs(E[:, c]))[::-1]
        if a[0] - a[1] <= 1e-6 * a[0]:
            out[:, c] *= np.sign(np.dot(V[:, c], E[:, c]))
    return out


def test_le_matches_oracle_c1():
    spec = CONFIGS["C1"]
    p, X, _ = gpu_problem(spec, "fp64")
    g = oracle_graph(spec, X)
    V, its, res = p.laplacian_eigenmap(spec.d, tol=1e-11)
    E = O.laplacian_eigenmap(g, spec.d)
    assert res <= 1e-11
    assert relerr(_align(V, E), E) <= 1e-7, relerr(_align(V, E), E)
    np.testing.assert_allclose(V.T @ (g.dvec[:, None] * V), np.eye(spec.d), atol=1e-10)
    np.testing.assert_allclose(V.T @ g.dvec, 0.0, atol=1e-9)
    p.close()


def test_le_path_graph_closed_form():
    from paper_1612_06496_gb300 import PFE
    ensure_built()
    n, d = 300, 4
    X = (0.3 * np.arange(n, dtype=np.float64))[:, None]
    a = np.arange(n - 1, dtype=np.int32)
    p = PFE(np.ascontiguousarray(X), sigma=0.5, edges=(a, a + 1), precision="fp64")
    V, its, res = p.laplacian_eigenmap(d, tol=1e-11)
    g = O.build_graph(X, a.astype(np.int64), (a + 1).astype(np.int64), 0.5)
    i = np.arange(n)
    E = np.stack([np.cos(np.pi * k * i / (n - 1)) for k in range(1, d + 1)], axis=1)
    E = E / np.sqrt(np.einsum("ic,i,ic->c", E, g.dvec, E))[None, :]
    E = E * np.sign(np.sum(V * E, axis=0))[None, :]  # the modes' ends tie in magnitude
    # eigenvector error <= residual / eigen-gap (Davis-Kahan): 1e-11 over the
    # smallest gap here (mu_5 - mu_4 ~ 5e-4) is ~2e-8 of a unit-D-norm vector
    assert np.max(np.abs(V - E)) <= 1e-6 * np.max(np.abs(E))
    p.close()


def test_le_k_components():
    """Three components (short chains with skip edges, so that the wanted
    eigenvalue 1 of D^{-1} W, multiplicity 3, is well apart from the next)."""
    from paper_1612_06496_gb300 import PFE
    ensure_built()
    rng = np.random.default_rng(6)
    sizes = [15, 22, 18]
    aa, bb, off, Xs = [], [], 0, []
    for s in sizes:
        Xs.append(rng.standard_normal((s, 2)) + 10 * len(Xs))
        for i in range(s - 1):
            aa.append(off + i)
            bb.append(off + i + 1)
        for i in range(0, s - 2, 2):
            aa.append(off + i)
            bb.append(off + i + 2)
        off += s
    X = np.ascontiguousarray(np.vstack(Xs))
    a, b = np.array(aa, dtype=np.int32), np.array(bb, dtype=np.int32)
    p = PFE(X, sigma=1.0, edges=(a, b), precision="fp64")
    V, its, res = p.laplacian_eigenmap(2, tol=1e-10)
    g = O.build_graph(X, a.astype(np.int64), b.astype(np.int64), 1.0)
    labels = np.repeat(np.arange(3), sizes)
    for c in range(2):
        for k in range(3):
            blk = V[labels == k, c]
            assert np.max(np.abs(blk - blk[0])) <= 1e-8 * np.max(np.abs(V))
    np.testing.assert_allclose(V.T @ g.dvec, 0.0, atol=1e-8)
    # same (degenerate) subspace as the oracle's
    E = O.laplacian_eigenmap(g, 2)
    Q = np.linalg.qr(np.sqrt(g.dvec)[:, None] * V)[0]
    R = np.sqrt(g.dvec)[:, None] * E
    assert np.linalg.norm(R - Q @ (Q.T @ R)) <= 1e-8 * np.linalg.norm(R)
    p.close()


def test_le_paper_scale_image():
    """481 x 321, radius 3 (C2 image), d = 8: the oracle's shift-invert route."""
    spec = CONFIGS["C2"]
    p, X, _ = gpu_problem(spec, "fp64")
    g = oracle_graph(spec, X)
    V, its, res = p.laplacian_eigenmap(spec.d, tol=1e-9, max_iter=2000, allow_notconv=True)
    E = O.laplacian_eigenmap(g, spec.d)
    np.testing.assert_allclose(V.T @ (g.dvec[:, None] * V), np.eye(spec.d), atol=1e-9)
    # compare the spanned subspaces (close eigenvalues may mix) and the vectors
    Q = np.linalg.qr(np.sqrt(g.dvec)[:, None] * V)[0]
    R = np.sqrt(g.dvec)[:, None] * E
    assert np.linalg.norm(R - Q @ (Q.T @ R)) <= 1e-5 * np.linalg.norm(R), (its, res)
    p.close()


def test_init_from_le_matches_oracle_trajectory():
    spec = CONFIGS["C1"]
    p, X, _ = gpu_problem(spec, "fp64", tol=1e-12)
    g = oracle_graph(spec, X)
    p.init(None, d=spec.d)
    info = p.info()
    assert info["le_residual"] <= 1e-9
    V0 = p.get("Y")
    E = O.laplacian_eigenmap(g, spec.d)
    assert relerr(_align(V0, E), E) <= 1e-6
    Y = np.empty_like(V0)
    p.solve(2, 3, Y, None)
    st = O.soc_pfe(g, E, 2, 3)
    # the iteration commutes with flipping a column's sign (Shrink is odd, the
    # polar factor of X S is polar(X) S): carry the starts' signs over
    sgn = np.sign(np.einsum("ic,i,ic->c", V0, g.dvec, E))
    assert relerr(Y * sgn[None, :], st.Y) <= 1e-5
    p.close()
