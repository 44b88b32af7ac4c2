"""Pins for the oracle's Laplacian-eigenmap start (generalised eigenvectors of
(D - W) v = mu D v, Sec. I) and its deterministic sign fix: closed forms,
a second library route, invariants and the k-component null space."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import pfe_oracle as O


def _path_graph(n, h=0.3, sigma=0.5):
    """Points on a line at equal spacing: every path edge has the same weight."""
    X = (h * np.arange(n, dtype=np.float64))[:, None]
    a = np.arange(n - 1)
    return O.build_graph(X, a, a + 1, sigma)


def _expected_path(n, d):
    """Path graph, uniform weights: mu_k = 1 - cos(pi k / (n-1)) with
    v_k(i) = cos(pi k i / (n-1)) (the discrete cosine modes), k = 1..d."""
    i = np.arange(n)
    return np.stack([np.cos(np.pi * k * i / (n - 1)) for k in range(1, d + 1)], axis=1)


@pytest.mark.parametrize("n", [40, 3200])  # dense route, shift-invert route
def test_path_graph_closed_form(n):
    d = 4
    g = _path_graph(n)
    V = O.laplacian_eigenmap(g, d)
    E = _expected_path(n, d)
    E = E / np.sqrt(np.einsum("ic,i,ic->c", E, g.dvec, E))[None, :]
    # the cosine modes are (anti)symmetric, so their largest entries tie at
    # both ends and rounding picks the sign: compare up to the sign here
    E = E * np.sign(np.sum(V * E, axis=0))[None, :]
    assert np.max(np.abs(V - E)) <= 1e-8 * np.max(np.abs(E))
    # the generalised eigen-equation with the closed-form eigenvalues
    L = (np.diag(g.dvec) - O.adjacency(g.n, g.a, g.b, g.w).toarray()) if n <= 100 else None
    if L is not None:
        for k in range(d):
            mu = 1 - np.cos(np.pi * (k + 1) / (n - 1))
            np.testing.assert_allclose(L @ V[:, k], mu * g.dvec * V[:, k], atol=1e-12)


def _random_connected(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 3))
    pairs = {(i, i + 1) for i in range(n - 1)}
    for _ in range(3 * n):
        i, j = sorted(rng.integers(0, n, 2))
        if i != j:
            pairs.add((int(i), int(j)))
    pairs = sorted(pairs)
    a = np.array([p[0] for p in pairs])
    b = np.array([p[1] for p in pairs])
    return O.build_graph(X, a, b, 0.9)


def test_normalised_laplacian_route_and_invariants():
    """Same subspace as the symmetric eigenproblem of I - D^{-1/2} W D^{-1/2}
    (v = D^{-1/2} u); V^T D V = I and V^T D 1 = 0."""
    g = _random_connected(120, 3)
    d = 5
    V = O.laplacian_eigenmap(g, d)
    Wm = O.adjacency(g.n, g.a, g.b, g.w).toarray()
    s = 1.0 / np.sqrt(g.dvec)
    Nl = np.eye(g.n) - s[:, None] * Wm * s[None, :]
    lam, U = sla.eigh(Nl)
    Vn = s[:, None] * U[:, 1:d + 1]
    assert np.all(np.diff(lam[:d + 2]) > 1e-6)  # simple eigenvalues: vectors unique up to sign
    np.testing.assert_allclose(np.abs(V), np.abs(Vn), atol=1e-9)
    np.testing.assert_allclose(V.T @ (g.dvec[:, None] * V), np.eye(d), atol=1e-11)
    np.testing.assert_allclose(V.T @ g.dvec, 0.0, atol=1e-11)
    # Rayleigh quotients ascend and equal the eigenvalues
    L = np.diag(g.dvec) - Wm
    np.testing.assert_allclose(np.einsum("ic,ij,jc->c", V, L, V), lam[1:d + 1], rtol=1e-9)


def test_sign_fix_is_deterministic():
    rng = np.random.default_rng(4)
    V = rng.standard_normal((30, 4))
    F = O.sign_fix(V)
    np.testing.assert_array_equal(O.sign_fix(-V), F)
    for c in range(4):
        assert F[np.argmax(np.abs(F[:, c])), c] > 0
    # a tie in magnitude: the smaller index decides
    T = np.zeros((5, 1))
    T[1, 0], T[3, 0] = -2.0, 2.0
    np.testing.assert_array_equal(O.sign_fix(T)[:, 0], [0, 2.0, 0, -2.0, 0])
    g = _random_connected(60, 8)
    V1 = O.laplacian_eigenmap(g, 3)
    np.testing.assert_array_equal(V1, O.laplacian_eigenmap(g, 3))


def test_k_components_null_space():
    """k components: mu = 0 has multiplicity k, so the first k-1 nontrivial
    eigenvectors are constant on every component (D-orthogonal to 1)."""
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
    g = O.build_graph(np.vstack(Xs), np.array(aa), np.array(bb), 1.0)
    V = O.laplacian_eigenmap(g, 2)
    labels = np.repeat(np.arange(3), sizes)
    for c in range(2):
        for k in range(3):
            blk = V[labels == k, c]
            assert np.max(np.abs(blk - blk[0])) <= 1e-10
    np.testing.assert_allclose(V.T @ g.dvec, 0.0, atol=1e-10)
