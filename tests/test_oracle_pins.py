"""Pins for the FP64 oracle: each test checks it against something other than
itself (closed forms, brute force, library routines, invariants, the paper's
printed numbers), so that a dropped term, a wrong sign or a transposed
operand in the oracle fails one of them."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import pfe_oracle as O

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _random_graph(n, p, seed, sigma=0.7, m=3):
    """Small random point cloud with an Erdos-Renyi edge set plus a path (connected)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, m))
    pairs = {(i, i + 1) for i in range(n - 1)}
    for i in range(n):
        for j in range(i + 1, n):
            if rng.uniform() < p:
                pairs.add((i, j))
    pairs = sorted(pairs)
    a = np.array([q[0] for q in pairs])
    b = np.array([q[1] for q in pairs])
    return X, a, b, sigma


# ---------------------------------------------------------------- graph


def test_stencil_offsets():
    # Sec. IV uses the 4-neighbourhood; the benchmark graphs use radius 2 and 3
    assert len(O.grid_offsets(1.0)) == 4
    assert len(O.grid_offsets(2.0)) == 12
    assert len(O.grid_offsets(3.0)) == 28
    for dx, dy in O.grid_offsets(3.0):
        assert 0 < dx * dx + dy * dy <= 9


def test_edge_counts_match_closed_form():
    with open(os.path.join(GOLD, "edge_counts.json")) as f:
        gold = json.load(f)
    for key in ("C1", "C2", "grid128_4nn"):
        g = gold[key]
        a, b = O.grid_edges(g["H"], g["W"], g["radius"])
        assert a.shape[0] == g["undirected"], key
        assert np.all(a < b)
        # no duplicates
        assert np.unique(a * g["n"] + b).shape[0] == a.shape[0]
    assert gold["C5"]["directed"] == 50290692


def test_paper_size_accounting():
    """Sec. III worked example: sizes of M, L, D~, W, Y and the dense inverse."""
    with open(os.path.join(GOLD, "size_accounting.json")) as f:
        g = json.load(f)
    H, W = g["image"]
    n, d = H * W, g["d"]
    MiB = 2 ** 20
    assert n * (n - 1) // 2 == g["M_rows"]
    assert n == g["M_cols"]
    # the paper counts 4 edge rows per vertex, 2 nonzeros per row of M
    assert 2 * 4 * n == g["M_nnz"]
    assert g["M_nnz"] * 8 / MiB == g["M_MB"]
    assert d * g["M_rows"] == g["L_rows"]                 # L = I_d (x) M (Eq. 3)
    assert d * n == g["L_cols"] == g["Dtilde_side"]       # D~ = I_d (x) D (Eq. 4)
    assert d * g["M_nnz"] == g["L_nnz"]
    assert g["L_nnz"] * 8 / MiB == g["L_MB"]
    assert d * n * 8 / MiB == g["Dtilde_MB"] == g["Y_MB"]
    assert 4 * n * 8 / MiB == g["W_MB"]
    assert (d * n) ** 2 * 8 / 2 ** 40 == g["inverse_TB"]
    # the exact 4-neighbourhood graph has fewer edges than the paper's 4n estimate
    a, b = O.grid_edges(H, W, 1.0)
    M = O.edge_operator(n, a, b, np.ones(a.shape[0]))
    assert M.shape == (2 * H * (W - 1), n)
    assert M.nnz == 2 * 2 * H * (W - 1) < g["M_nnz"]


def test_heat_kernel_closed_form():
    sigma = 0.3
    X = np.array([[0.0, 0.0, 0.0], [sigma, 0.0, 0.0], [0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    w = O.heat_kernel_weights(X, np.array([0, 0, 0]), np.array([1, 2, 3]), sigma)
    assert w[0] == pytest.approx(np.exp(-0.5), rel=1e-15)
    assert w[1] == 1.0
    assert w[2] == pytest.approx(np.exp(-25.0 / (2 * sigma * sigma)), rel=1e-13)


def test_system_matrix_and_lambda_on_a_path():
    """Three points on a line, edges 0-1 and 1-2: every entry of
    A = lam (D2 - W o W) + r D and lam = sqrt(vol W) written out by hand."""
    sigma = 0.5
    X = np.array([[0.0, 0.0], [0.3, 0.0], [0.3, 0.8]])
    w1, w2 = np.exp(-0.09 / (2 * sigma ** 2)), np.exp(-0.64 / (2 * sigma ** 2))
    g = O.build_graph(X, np.array([0, 1]), np.array([1, 2]), sigma, r=0.7)
    lam, r = np.sqrt(2.0 * (w1 + w2)), 0.7        # vol W counts each edge from both ends
    assert g.lam == pytest.approx(lam, rel=1e-15)
    expect = np.array([[lam * w1 ** 2 + r * w1, -lam * w1 ** 2, 0.0],
                       [-lam * w1 ** 2, lam * (w1 ** 2 + w2 ** 2) + r * (w1 + w2), -lam * w2 ** 2],
                       [0.0, -lam * w2 ** 2, lam * w2 ** 2 + r * w2]])
    np.testing.assert_allclose(g.A.toarray(), expect, rtol=1e-14, atol=0.0)
    # an explicit lambda is kept as given
    assert O.build_graph(X, np.array([0, 1]), np.array([1, 2]), sigma, lam=2.5).lam == 2.5


def test_degrees_and_edge_operator_laplacian():
    """M^T M is the Laplacian of the squared weights; d is the row sum of W."""
    X, a, b, sigma = _random_graph(9, 0.4, 3)
    n = X.shape[0]
    w = O.heat_kernel_weights(X, a, b, sigma)
    Wd = np.zeros((n, n))
    for k in range(a.shape[0]):   # brute force, one pair at a time
        Wd[a[k], b[k]] = Wd[b[k], a[k]] = np.exp(-np.sum((X[a[k]] - X[b[k]]) ** 2) / (2 * sigma ** 2))
    dvec = O.degrees(O.adjacency(n, a, b, w))
    np.testing.assert_allclose(dvec, Wd.sum(axis=1), rtol=1e-14)
    M = O.edge_operator(n, a, b, w).toarray()
    W2 = Wd * Wd
    lap = np.diag(W2.sum(axis=1)) - W2
    np.testing.assert_allclose(M.T @ M, lap, atol=1e-14)
    # each row of M: +w at the first endpoint, -w at the second
    for k in range(a.shape[0]):
        assert M[k, a[k]] == pytest.approx(w[k]) and M[k, b[k]] == pytest.approx(-w[k])
        assert np.count_nonzero(M[k]) == 2


# ---------------------------------------------------------------- shrink


def test_shrink_closed_form_and_prox():
    g = 0.25
    y = np.array([-1.0, -0.25, -0.1, -0.0, 0.0, 0.1, 0.25, 0.26, 1.0, 3 * 0.25])
    z = O.shrink(y, g)
    np.testing.assert_array_equal(z, [-0.75, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.26 - 0.25, 0.75, 0.5])
    assert np.isnan(O.shrink(np.array([np.nan]), g)[0])
    # subnormals: below any positive threshold they shrink to zero; with
    # gamma = 0 Shrink is the identity on them
    tiny = np.array([5e-324, -5e-324, 2.2e-308, -1e-310])
    np.testing.assert_array_equal(O.shrink(tiny, g), np.zeros(4))
    np.testing.assert_array_equal(O.shrink(tiny, 0.0), tiny)
    assert O.shrink(np.array([1e-310]), 1e-310)[0] == 0.0
    assert O.shrink(np.array([3e-310]), 1e-310)[0] == 3e-310 - 1e-310
    # odd function
    rng = np.random.default_rng(0)
    v = rng.standard_normal(1000)
    np.testing.assert_array_equal(O.shrink(-v, g), -O.shrink(v, g))
    # Shrink is the proximal map of gamma*|z|: brute-force minimisation on a grid
    grid = np.linspace(-3, 3, 600001)
    for yy in rng.uniform(-2, 2, 25):
        f = g * np.abs(grid) + 0.5 * (grid - yy) ** 2
        assert abs(grid[np.argmin(f)] - O.shrink(np.array([yy]), g)[0]) < 2e-5


# ------------------------------------------------- compact vs Kronecker forms


def _kron_setup(seed=5, n=8, d=3):
    X, a, b, sigma = _random_graph(n, 0.35, seed)
    g = O.build_graph(X, a, b, sigma, lam=1.7, r=0.9)
    rng = np.random.default_rng(seed + 1)
    Y = rng.standard_normal((n, d))
    return g, Y, rng


def vec(Z):
    return Z.reshape(-1, order="F")


def test_vec_identities_eq7_8_11_12():
    g, Y, _ = _kron_setup()
    d = Y.shape[1]
    M = g.M.toarray()
    L = np.kron(np.eye(d), M)                   # Eq. 3
    Dt = np.kron(np.eye(d), np.diag(g.dvec))    # Eq. 4
    np.testing.assert_allclose(L @ vec(Y), vec(M @ Y), atol=1e-13)                    # Eq. 7
    np.testing.assert_allclose(np.sqrt(Dt) @ vec(Y), vec(np.sqrt(g.dvec)[:, None] * Y), atol=1e-13)  # Eq. 8
    np.testing.assert_allclose(L.T @ L @ vec(Y), vec(M.T @ M @ Y), atol=1e-12)          # Eq. 11
    np.testing.assert_allclose(Dt @ vec(Y), vec(g.dvec[:, None] * Y), atol=1e-13)      # Eq. 12


def test_normal_equations_solve_least_squares_and_sign_of_q2():
    """The compact solve (Eq. 13, Q2 = P - B) minimises Alg. 2 step 5's objective.

    Independent route: numpy lstsq on the stacked least-squares system
    [sqrt(lam) M; sqrt(r) D^{1/2}] Y ~ [sqrt(lam)(d - b); sqrt(r)(P - B)].
    The paper's printed sign (Q2 = B - P) fails this test.
    """
    g, Y0, rng = _kron_setup(seed=11)
    n, d = Y0.shape
    E = g.n_edges
    st = O.init_state(g, Y0)
    st.B = 0.1 * rng.standard_normal((n, d))
    st.bs = 0.05 * rng.standard_normal((E, d))
    st.ds = 0.05 * rng.standard_normal((E, d))
    bs0, ds0 = st.bs.copy(), st.ds.copy()
    O.split_bregman_step(g, st, O.DirectSolver(g.A))
    sq = np.sqrt(g.dvec)[:, None]
    K = np.vstack([np.sqrt(g.lam) * g.M.toarray(), np.sqrt(g.r) * np.diag(sq[:, 0])])
    rhs = np.vstack([np.sqrt(g.lam) * (ds0 - bs0), np.sqrt(g.r) * (st.P - st.B)])
    Yls = np.linalg.lstsq(K, rhs, rcond=None)[0]
    np.testing.assert_allclose(st.Y, Yls, rtol=1e-10, atol=1e-12)
    # the Kronecker form (Eq. 6) with q2 = P_v - B_v gives the same Y (Eq. 13)
    Md = g.M.toarray()
    L = np.kron(np.eye(d), Md)
    Dt = np.kron(np.eye(d), np.diag(g.dvec))
    lhs = 0.5 * g.lam * L.T @ L + 0.5 * g.r * Dt
    q1 = vec(ds0 - bs0)
    q2 = vec(st.P - st.B)
    yv = np.linalg.solve(lhs, 0.5 * g.lam * L.T @ q1 + 0.5 * g.r * np.sqrt(Dt) @ q2)
    np.testing.assert_allclose(st.Y, yv.reshape(n, d, order="F"), rtol=1e-10, atol=1e-12)
    # with the sign as printed the solution is not the minimiser
    yv_bad = np.linalg.solve(lhs, 0.5 * g.lam * L.T @ q1 - 0.5 * g.r * np.sqrt(Dt) @ q2)
    assert np.linalg.norm(yv_bad - vec(Yls)) > 1e-3 * np.linalg.norm(Yls)


def test_compact_trajectory_equals_kronecker_alg2():
    """Alg. 2 run literally on L, D~ (dense, vectorised, Eqs. 3-6) equals the
    compact oracle (Eqs. 9, 10, 13) over several inner iterations."""
    g, Y0, rng = _kron_setup(seed=21, n=9, d=2)
    n, d = Y0.shape
    st = O.init_state(g, Y0)
    st.B = 0.2 * rng.standard_normal((n, d))
    P_v, B_v = vec(st.P), vec(st.B)
    Md = g.M.toarray()
    L = np.kron(np.eye(d), Md)
    Dt = np.kron(np.eye(d), np.diag(g.dvec))
    lhs = 0.5 * g.lam * L.T @ L + 0.5 * g.r * Dt
    b_l = np.zeros(L.shape[0])
    d_l = np.zeros(L.shape[0])
    solve = O.DirectSolver(g.A)
    for _ in range(4):
        yv = np.linalg.solve(lhs, 0.5 * g.lam * L.T @ (d_l - b_l) + 0.5 * g.r * np.sqrt(Dt) @ (P_v - B_v))
        Ly = L @ yv
        d_new = np.sign(Ly + b_l) * np.maximum(np.abs(Ly + b_l) - 1.0 / g.lam, 0.0)
        b_l = b_l + Ly - d_new
        d_l = d_new
        O.split_bregman_step(g, st, solve)
        np.testing.assert_allclose(st.Y, yv.reshape(n, d, order="F"), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(st.bs, b_l.reshape(-1, d, order="F"), atol=1e-11)
        np.testing.assert_allclose(st.ds, d_l.reshape(-1, d, order="F"), atol=1e-11)


# ---------------------------------------------------------------- solves


def test_direct_dense_and_pcg_agree():
    X, a, b, sigma = _random_graph(30, 0.15, 7)
    g = O.build_graph(X, a, b, sigma)
    rng = np.random.default_rng(8)
    rhs = rng.standard_normal((g.n, 4))
    Yd = np.linalg.solve(g.A.toarray(), rhs)
    Ylu, _ = O.DirectSolver(g.A)(rhs)
    Ypcg, info = O.jacobi_pcg(g.A, rhs, np.zeros_like(rhs), tol=1e-14, max_iter=1000)
    np.testing.assert_allclose(Ylu, Yd, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(Ypcg, Yd, rtol=1e-9, atol=1e-12)
    assert info["converged"]
    assert np.all(info["true_relres"] < 1e-12)


def test_pcg_matches_scipy_cg_and_counts():
    """Per-column Jacobi PCG == scipy's preconditioned CG solution; columns are independent."""
    import scipy.sparse.linalg as spla
    X, a, b, sigma = _random_graph(60, 0.08, 9)
    g = O.build_graph(X, a, b, sigma)
    rng = np.random.default_rng(10)
    rhs = rng.standard_normal((g.n, 3))
    Y, info = O.jacobi_pcg(g.A, rhs, np.zeros_like(rhs), tol=1e-10, max_iter=500, refresh=0)
    Minv = spla.LinearOperator(g.A.shape, matvec=lambda v: v / g.A.diagonal())
    for c in range(3):
        ref, ok = spla.cg(g.A, rhs[:, c], rtol=1e-12, maxiter=2000, M=Minv)
        np.testing.assert_allclose(Y[:, c], ref, rtol=1e-7, atol=1e-9)
        yc, ic = O.jacobi_pcg(g.A, rhs[:, c:c + 1], np.zeros((g.n, 1)), tol=1e-10, max_iter=500, refresh=0)
        assert ic["iters"][0] == info["iters"][c]
        np.testing.assert_allclose(yc[:, 0], Y[:, c], rtol=1e-12, atol=1e-14)
    # warm start at the solution converges immediately
    _, info2 = O.jacobi_pcg(g.A, rhs, Y, tol=1e-8, max_iter=500)
    assert np.all(info2["iters"] == 0)


# ---------------------------------------------------------------- P-step


def test_polar_factor_procrustes():
    rng = np.random.default_rng(12)
    Xm = rng.standard_normal((50, 5))
    P = O.polar_factor(Xm)
    np.testing.assert_allclose(P.T @ P, np.eye(5), atol=1e-14)
    U, _ = sla.polar(Xm)                               # library polar decomposition
    np.testing.assert_allclose(P, U, atol=1e-13)
    # X (X^T X)^{-1/2} through a symmetric eigendecomposition gives the same matrix
    lam, V = np.linalg.eigh(Xm.T @ Xm)
    np.testing.assert_allclose(P, Xm @ (V / np.sqrt(lam)) @ V.T, atol=1e-12)
    # Procrustes optimality against random orthonormal matrices
    best = np.linalg.norm(P - Xm)
    for _ in range(1000):
        Q, _ = np.linalg.qr(rng.standard_normal((50, 5)))
        assert np.linalg.norm(Q - Xm) >= best - 1e-12
    with pytest.raises(np.linalg.LinAlgError):
        O.polar_factor(np.ones((10, 2)))


# ---------------------------------------------------------------- whole loop


def _c1_like(H=12, W=14, seed=3, d=3):
    from synth import ImageSpec, make_problem
    spec = ImageSpec("t", H, W, 3, 0.05, seed=seed, radius=2.0, sigma=0.1, d=d)
    X, Y0 = make_problem(spec)
    g = O.build_grid_graph(X, H, W, 2.0, 0.1)
    return g, Y0


def test_constraint_holds_after_every_p_step():
    g, Y0 = _c1_like()
    st = O.init_state(g, Y0)
    np.testing.assert_allclose(st.Y.T @ (g.dvec[:, None] * st.Y), np.eye(3), atol=1e-12)
    solve = O.DirectSolver(g.A)
    for _ in range(4):
        O.reset_inner(st)
        for _ in range(3):
            O.split_bregman_step(g, st, solve)
        O.p_and_b_step(g, st)
        Yh = O.embedding(g, st)
        assert np.max(np.abs(Yh.T @ (g.dvec[:, None] * Yh) - np.eye(3))) <= 1e-10


def test_disconnected_components_fixed_point():
    """k components + a D-orthonormal piecewise-constant start is a fixed point:
    M Y = 0, so Z = b = 0, the solve returns Y, and the polar step returns P."""
    rng = np.random.default_rng(13)
    sizes = [7, 9, 6]
    X_parts, aa, bb, off = [], [], [], 0
    for s in sizes:
        X_parts.append(rng.standard_normal((s, 3)) + 10 * off)
        for i in range(s - 1):
            aa.append(off + i)
            bb.append(off + i + 1)
        aa.append(off)
        bb.append(off + s - 1)
        off += s
    X = np.vstack(X_parts)
    g = O.build_graph(X, np.array(aa), np.array(bb), 1.5)
    labels = np.repeat(np.arange(3), sizes)
    ind = np.stack([(labels == k).astype(float) for k in range(3)], axis=1)
    Y0 = ind[:, :2] - 0.3 * ind[:, 2:3]
    st = O.soc_pfe(g, Y0, n_outer=3, n_inner=3)
    Yi = O.d_orthonormalize(Y0, g.dvec)
    np.testing.assert_allclose(st.Y, Yi, atol=1e-12)
    np.testing.assert_allclose(O.embedding(g, st), Yi, atol=1e-12)
    for k in range(3):
        blk = st.Y[labels == k]
        assert np.max(np.abs(blk - blk[0])) <= 1e-12
    assert np.max(np.abs(st.B)) <= 1e-12


def test_soc_with_pcg_matches_direct():
    g, Y0 = _c1_like(seed=4)
    st_d = O.soc_pfe(g, Y0, n_outer=2, n_inner=3, solver="direct")
    st_p = O.soc_pfe(g, Y0, n_outer=2, n_inner=3, solver="pcg", tol=1e-13)
    rel = np.linalg.norm(st_p.Y - st_d.Y) / np.linalg.norm(st_d.Y)
    assert rel < 1e-9


def test_zero_degree_vertex_rejected():
    X = np.zeros((4, 2))
    with pytest.raises(ValueError):
        O.build_graph(X, np.array([0, 1]), np.array([1, 2]), 1.0)


def test_two_stage_stage2_minimises_the_relaxed_y_problem():
    """Stage II (Sec. IV) runs Alg. 2 with P, B held: its iterates approach
    the minimiser of |MY|_1 + (r/2 lam) ... the Y-step objective of Alg. 2
    step 5 with P, B fixed.  Split Bregman for that convex problem converges,
    so after many iterations the objective is below its value at Stage I's Y
    and at random perturbations of the result."""
    X, a, b, sigma = _random_graph(40, 0.15, 21)
    g = O.build_graph(X, a, b, sigma)
    rng = np.random.default_rng(2)
    Y0 = rng.standard_normal((g.n, 3))
    st1 = O.soc_pfe(g, Y0, 3, 4)
    st2 = O.two_stage(g, Y0, 3, 4, 400)
    np.testing.assert_allclose(st2.P, st1.P)          # P, B held in Stage II
    np.testing.assert_allclose(st2.B, st1.B)
    sq = np.sqrt(g.dvec)[:, None]

    def f(Y):  # the Y-step objective (Alg. 2 step 5; Eq. 5 in compact form)
        return np.abs(g.M @ Y).sum() + 0.5 * g.r * np.sum((sq * Y - st1.P + st1.B) ** 2)

    f2 = f(st2.Y)
    assert f2 <= f(st1.Y) + 1e-12
    for _ in range(20):
        assert f2 <= f(st2.Y + 1e-3 * rng.standard_normal(st2.Y.shape)) + 1e-12


def test_edge_count_fixture_is_what_its_script_writes():
    """tests/golden/edge_counts.json is the closed-form output of
    tests/golden/make_edge_counts.py, entry for entry."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_edge_counts", os.path.join(GOLD, "make_edge_counts.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(GOLD, "edge_counts.json")) as f:
        gold = json.load(f)
    shapes = {"C1": (32, 32, 2.0), "C2": (481, 321, 3.0), "C5": (2048, 2048, 2.0), "grid128_4nn": (128, 128, 1.0)}
    assert set(gold) == set(shapes)
    for key, (W, H, R) in shapes.items():
        assert mod.counts(W, H, R) == gold[key], key
