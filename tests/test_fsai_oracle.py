"""Pins of the learned-FSAI oracle: finite differences for every gradient,
the untrained network equals Jacobi, and the Kaporin gradient vanishes at
classical FSAI (the known minimiser over the same pattern)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fsai_oracle as F
from oracle import pfe_oracle as O
from synth import ImageSpec, make_problem


def _tiny_graph(H=6, W=6, radius=2.0, seed=3):
    spec = ImageSpec("t", H, W, 3, 0.05, seed=seed, radius=radius, sigma=0.1, d=2)
    X, _ = make_problem(spec)
    return O.build_grid_graph(X, H, W, radius, 0.1)


def test_untrained_network_is_jacobi():
    g = _tiny_graph()
    th = F.init_params(1)
    Fd, Fe = F.entry_features(g)
    od, _ = F.mlp_forward(th, Fd)
    oe, _ = F.mlp_forward(th, Fe)
    G, gd, ge = F.assemble_G(g, od, oe)
    Ad = g.A.diagonal()
    np.testing.assert_allclose(gd, 1.0 / np.sqrt(Ad), rtol=1e-15)
    assert np.all(ge == 0.0)
    R = np.random.default_rng(0).standard_normal((g.n, 3))
    np.testing.assert_allclose(F.fsai_apply(G, R), R / Ad[:, None], rtol=1e-13)


def test_features_definition():
    g = _tiny_graph()
    Fd, Fe = F.entry_features(g)
    Ad = g.A.diagonal()
    k = 7
    a, b = g.a[k], g.b[k]
    assert Fe[k, 0] == pytest.approx(g.lam * g.w[k] ** 2 / np.sqrt(Ad[a] * Ad[b]), rel=1e-14)
    assert Fe[k, 1] == pytest.approx(g.r * g.dvec[b] / Ad[b], rel=1e-14)
    assert Fe[k, 2] == pytest.approx(g.r * g.dvec[a] / Ad[a], rel=1e-14)
    i = 20
    lower = g.b == i
    assert Fd[i, 0] == pytest.approx(np.sum(Fe[lower, 0] ** 2), rel=1e-13)
    # rho lies in (0, 1): the Jacobi-scaled coupling of an M-matrix row
    assert np.all(Fe[:, 0] > 0) and np.all(Fe[:, 0] < 1)


def test_kaporin_gradient_matches_finite_differences():
    g = _tiny_graph(5, 5)
    G0 = F.classical_fsai(g.A)
    rng = np.random.default_rng(2)
    G = G0.copy()
    G.data = G.data * (1 + 0.1 * rng.standard_normal(G.data.shape))
    L, dG, _ = F.kaporin(g, G)
    dG = dG.tocsr()
    Gc = G.tocoo()
    for t in rng.choice(Gc.nnz, 15, replace=False):
        i, j = Gc.row[t], Gc.col[t]
        # central differences: rounding ~eps*|L|/h plus truncation ~h^2, both
        # well below 1e-5 relative at this step
        h = 1e-5 * max(abs(Gc.data[t]), 1e-3)
        Gp = G.tolil(); Gp[i, j] += h
        Gm = G.tolil(); Gm[i, j] -= h
        fd = (F.kaporin(g, Gp.tocsr())[0] - F.kaporin(g, Gm.tocsr())[0]) / (2 * h)
        assert fd == pytest.approx(dG[i, j], rel=1e-5, abs=1e-9)


def test_kaporin_stationary_at_classical_fsai():
    """Classical FSAI minimises the Kaporin number over the pattern, so the
    gradient vanishes there and tr(G A G^T) = n."""
    g = _tiny_graph(7, 6)
    G = F.classical_fsai(g.A)
    L, dG, T = F.kaporin(g, G)
    assert T == pytest.approx(g.n, rel=1e-12)
    assert np.max(np.abs(dG.toarray())) < 1e-12
    # and it beats Jacobi and perturbations of itself
    Lj = F.kaporin(g, sp.diags(1.0 / np.sqrt(g.A.diagonal())).tocsr())[0]
    assert L < Lj
    rng = np.random.default_rng(4)
    for _ in range(5):
        Gp = G.copy()
        Gp.data = Gp.data * (1 + 0.05 * rng.standard_normal(Gp.data.shape))
        assert F.kaporin(g, Gp)[0] > L


def test_network_gradient_matches_finite_differences():
    g = _tiny_graph(6, 6)
    th = F.init_params(5)
    rng = np.random.default_rng(6)
    th = th + 0.05 * rng.standard_normal(th.shape)   # away from the all-zero output layer
    L, grad, _ = F.loss_and_grad(th, g)
    for k in rng.choice(F.NPARAM, 25, replace=False):
        h = 1e-6
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        fd = (F.loss_and_grad(tp, g)[0] - F.loss_and_grad(tm, g)[0]) / (2 * h)
        assert fd == pytest.approx(grad[k], rel=1e-5, abs=1e-9), k


def test_classical_fsai_reduces_pcg_iterations():
    g = _tiny_graph(24, 24)
    rng = np.random.default_rng(7)
    Bm = rng.standard_normal((g.n, 2))
    dinv = 1.0 / g.A.diagonal()
    G = F.classical_fsai(g.A)

    def pcg(Minv):
        X = np.zeros_like(Bm); R = Bm.copy(); Z = Minv(R); P = Z.copy(); rz = (R * Z).sum(0)
        for it in range(1, 2000):
            Q = g.A @ P; al = rz / (P * Q).sum(0); X += al * P; R -= al * Q
            if np.max(np.linalg.norm(R, axis=0) / np.linalg.norm(Bm, axis=0)) < 1e-8:
                return it
            Z = Minv(R); rzn = (R * Z).sum(0); P = Z + rzn / rz * P; rz = rzn
        return 2000
    assert pcg(lambda R: F.fsai_apply(G, R)) < pcg(lambda R: dinv[:, None] * R)


def test_oracle_pcg_exact_preconditioner_takes_one_step():
    """With M^-1 = A^-1 the first direction is the whole error, alpha = 1 and
    every column converges after one iteration (any start); with M = I the
    residual norms of CG on a 1-dimensional Krylov space match the closed form
    of steepest descent."""
    g = _tiny_graph(9, 8)
    rng = np.random.default_rng(5)
    Bm = rng.standard_normal((g.n, 3))
    X0 = rng.standard_normal((g.n, 3))
    solve = O.DirectSolver(g.A)
    X, info = O.pcg(g.A, Bm, X0, 1e-10, 50, 0, lambda R: solve(R)[0])
    assert info["converged"] and np.all(info["iters"] == 1)
    np.testing.assert_allclose(X, solve(Bm)[0], rtol=1e-9, atol=1e-12)
    # one identity-preconditioned step: x1 = x0 + (r.r / r.A r) r
    X1, _ = O.pcg(g.A, Bm, X0, 0.0, 1, 0, lambda R: R)
    R0 = Bm - g.A @ X0
    al = (R0 * R0).sum(0) / (R0 * (g.A @ R0)).sum(0)
    np.testing.assert_allclose(X1, X0 + al * R0, rtol=1e-12)


def test_oracle_pcg_with_fsai_matches_direct_solve():
    g = _tiny_graph(20, 18, radius=3.0)
    Bm = np.random.default_rng(8).standard_normal((g.n, 2))
    G = F.classical_fsai(g.A)
    X, info = O.pcg(g.A, Bm, np.zeros_like(Bm), 1e-10, 2000, 50, lambda R: F.fsai_apply(G, R))
    _, ij = O.jacobi_pcg(g.A, Bm, np.zeros_like(Bm), 1e-10, 2000)
    assert info["converged"] and info["iters"].max() < ij["iters"].max()
    np.testing.assert_allclose(X, O.DirectSolver(g.A)(Bm)[0], rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("H,W,radius,seed", [(40, 48, 2.0, 11), (32, 40, 3.0, 12)])
def test_trained_network_cuts_pcg_iterations(H, W, radius, seed):
    """What the trained network (the committed weights) gains over the method
    without it, on images it was not trained on: through the oracle's network
    and PCG, the learned factor needs at most 0.7x the Jacobi iterations to
    rel-res 1e-6 and about as many as classical FSAI, the optimum of its
    pattern (measured: 0.54x and 0.59x Jacobi, 1.0x and 0.97x classical)."""
    from paper_1612_06496_gb300.learned import load_weights
    spec = ImageSpec("t", H, W, 4, 0.05, seed=seed, radius=radius, sigma=0.1, d=4)
    X, _ = make_problem(spec)
    g = O.build_grid_graph(X, H, W, radius, 0.1)
    th = load_weights().astype(np.float64)
    Fd, Fe = F.entry_features(g)
    od, _ = F.mlp_forward(th, Fd)
    oe, _ = F.mlp_forward(th, Fe)
    G, _, _ = F.assemble_G(g, od, oe)
    Gc = F.classical_fsai(g.A)
    R = np.random.default_rng(31).standard_normal((g.n, 4))
    z = np.zeros_like(R)
    _, ij = O.jacobi_pcg(g.A, R, z, 1e-6, 5000)
    Xl, il = O.pcg(g.A, R, z, 1e-6, 5000, 50, lambda Q: F.fsai_apply(G, Q))
    _, ic = O.pcg(g.A, R, z, 1e-6, 5000, 50, lambda Q: F.fsai_apply(Gc, Q))
    n_j, n_l, n_c = ij["iters"].max(), il["iters"].max(), ic["iters"].max()
    assert il["converged"] and n_l <= 0.7 * n_j, (n_l, n_j)
    assert n_l <= 1.1 * n_c, (n_l, n_c)
    Xd = O.DirectSolver(g.A)(R)[0]
    assert np.linalg.norm(Xl - Xd) <= 1e-4 * np.linalg.norm(Xd)


def test_adam_moves_by_lr_sign_of_a_constant_gradient():
    """Adam's bias corrections make both moment estimates exact when the
    gradient is constant, so every step moves a parameter by
    lr g / (|g| + eps): about lr against the sign of its gradient, whatever
    the gradient's scale."""
    rng = np.random.default_rng(3)
    g = rng.choice([-1.0, 1.0], 60) * np.logspace(-3, 3, 60)
    th0 = rng.standard_normal(60)
    th, m, v = th0.copy(), np.zeros(60), np.zeros(60)
    for step in range(1, 21):
        th, m, v = F.adam_step(th, g, m, v, step, lr=0.01)
    np.testing.assert_allclose(th, th0 - 20 * 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)
    # no gradient, no moments: no movement
    th2, _, _ = F.adam_step(th0, np.zeros(60), np.zeros(60), np.zeros(60), 1, lr=0.01)
    np.testing.assert_array_equal(th2, th0)


def test_adam_moments_are_the_weighted_sums_of_past_gradients():
    """After T steps m = (1 - b1) sum_k b1^(T-k) g_k and v likewise with g_k^2
    (the recursion unrolled); the T-th step is lr mhat / (sqrt(vhat) + eps)."""
    rng = np.random.default_rng(4)
    T, n, lr, b1, b2, eps = 6, 40, 3e-3, 0.8, 0.95, 1e-6
    gs = rng.standard_normal((T, n))
    th, m, v = rng.standard_normal(n), np.zeros(n), np.zeros(n)
    for t in range(1, T + 1):
        prev = th
        th, m, v = F.adam_step(th, gs[t - 1], m, v, t, lr, b1, b2, eps)
    w1 = (1 - b1) * b1 ** np.arange(T - 1, -1, -1)
    w2 = (1 - b2) * b2 ** np.arange(T - 1, -1, -1)
    m_sum, v_sum = w1 @ gs, w2 @ gs ** 2
    np.testing.assert_allclose(m, m_sum, rtol=1e-13)
    np.testing.assert_allclose(v, v_sum, rtol=1e-13)
    last = lr * (m_sum / (1 - b1 ** T)) / (np.sqrt(v_sum / (1 - b2 ** T)) + eps)
    np.testing.assert_allclose(prev - th, last, rtol=1e-12, atol=1e-15)  # prev - th cancels: |theta| ~ 1


# ---------------------------------------------------------------- the network itself


def _theta_random(seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(F.NPARAM) * 0.3


def _torch_mlp(theta):
    """The same network as torch.nn layers in FP64 (Linear computes x W^T + b,
    so each weight is the transpose of the oracle's row-major W)."""
    torch = pytest.importorskip("torch")
    W1, b1, W2, b2, W3, b3 = F.unpack(theta)
    net = torch.nn.Sequential(torch.nn.Linear(4, F.H), torch.nn.ReLU(), torch.nn.Linear(F.H, F.H), torch.nn.ReLU(),
                              torch.nn.Linear(F.H, 2)).double()
    with torch.no_grad():
        for layer, W, b in ((net[0], W1, b1), (net[2], W2, b2), (net[4], W3, b3)):
            layer.weight.copy_(torch.from_numpy(np.ascontiguousarray(W.T)))
            layer.bias.copy_(torch.from_numpy(b))
    return torch, net


def test_mlp_forward_matches_torch_nn():
    """mlp_forward against torch.nn's Linear/ReLU stack in FP64, on inputs of
    both signs (both ReLUs cut)."""
    theta = _theta_random(1)
    Fm = np.random.default_rng(2).standard_normal((300, 4)) * 2.0
    out, _ = F.mlp_forward(theta, Fm)
    torch, net = _torch_mlp(theta)
    ref = net(torch.from_numpy(Fm)).detach().numpy()
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_mlp_backward_matches_torch_autograd():
    """mlp_backward (the gradient of sum(out * dout) w.r.t. the parameters)
    against torch's autograd of the same network in FP64."""
    theta = _theta_random(3)
    rng = np.random.default_rng(4)
    Fm = rng.standard_normal((200, 4)) * 2.0
    dout = rng.standard_normal((200, 2))
    _, cache = F.mlp_forward(theta, Fm)
    g = F.mlp_backward(theta, cache, dout)
    torch, net = _torch_mlp(theta)
    (net(torch.from_numpy(Fm)) * torch.from_numpy(dout)).sum().backward()
    parts = [net[0].weight.grad.T, net[0].bias.grad, net[2].weight.grad.T, net[2].bias.grad, net[4].weight.grad.T,
             net[4].bias.grad]
    ref = np.concatenate([np.ascontiguousarray(p.numpy()).ravel() for p in parts])
    np.testing.assert_allclose(g, ref, rtol=1e-11, atol=1e-12)


def test_mlp_forward_worked_by_hand():
    """A network whose output follows by hand.  W1 copies the four inputs to
    units 0..3; W2 shifts unit k to unit k + 1 (not symmetric, so a transposed
    W2 reads unit k + 1 instead) and also sends -h1_1 to unit 10; b2 = -0.5
    makes the second ReLU cut.  Input (1, -2, 3, 0.5): h1 = (1, 0, 3, 0.5)
    (the first ReLU cuts -2; without it unit 10 would get 2 - 0.5 and out0
    1.5 more); a2_j = h1_{j-1} - 0.5, so h2 = (0, 0.5, 0, 2.5, 0, ...);
    out0 = 0.5 * 2 + 2.5 * 4 + 0.25 = 11.25 and out1 = 2.5 * 1 - 1 = 1.5."""
    W1 = np.zeros((4, F.H))
    W1[np.arange(4), np.arange(4)] = 1.0
    W2 = np.zeros((F.H, F.H))
    W2[np.arange(F.H - 1), np.arange(1, F.H)] = 1.0
    W2[1, 10] = -1.0
    b2 = np.full(F.H, -0.5)
    W3 = np.zeros((F.H, 2))
    W3[:4, 0] = [1.0, 2.0, 3.0, 4.0]
    W3[10, 0] = 1.0
    W3[3, 1] = 1.0
    theta = np.concatenate([W1.ravel(), np.zeros(F.H), W2.ravel(), b2, W3.ravel(), [0.25, -1.0]])
    out, _ = F.mlp_forward(theta, np.array([[1.0, -2.0, 3.0, 0.5]]))
    np.testing.assert_allclose(out, [[11.25, 1.5]], rtol=0, atol=1e-15)


def test_bf16_rounding_matches_torch():
    """bf16_round (nearest, ties to even, via FP32) against torch's bfloat16
    conversion, ties and a boundary included: 1 + 2^-8 is a tie between 1
    and 1 + 2^-7 and rounds to the even 1; 1 + 3 * 2^-8 rounds to 1 + 2^-6."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.integers(-6, 6, 1000),
                        [1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 0.0, 2.0 ** -126]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(F.bf16_round(x), ref)
    assert F.bf16_round(1 + 2.0 ** -8) == 1.0 and F.bf16_round(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6


def test_bf16_network_stays_within_bf16_rounding_of_fp64():
    """The BF16 emulation of the hidden layer moves the outputs by about the
    BF16 unit (2^-8 relative per operand) and no more."""
    theta = _theta_random(5)
    Fm = np.random.default_rng(6).standard_normal((500, 4))
    o64, _ = F.mlp_forward(theta, Fm)
    o16, _ = F.mlp_forward(theta, Fm, bf16=True)
    rel = np.linalg.norm(o16 - o64) / np.linalg.norm(o64)
    assert 1e-5 < rel < 2e-2, rel


# ---- the right-hand-side residual term of the training criterion

def test_rhs_residual_one_by_one_closed_form():
    """n = 1: A = [a], G = [g], b = [beta] give R = (a g^2 - 1)^2 and
    dR/dg = 4 a g (a g^2 - 1), whatever beta."""
    from types import SimpleNamespace
    for a, gv, beta in ((3.0, 0.4, 2.0), (0.5, 1.7, -0.3), (2.0, 2 ** -0.5, 5.0)):
        g = SimpleNamespace(A=sp.csr_matrix([[a]]))
        R, dR = F.rhs_residual(g, sp.csr_matrix([[gv]]), np.array([[beta]]))
        assert R == pytest.approx((a * gv * gv - 1) ** 2, rel=1e-14, abs=1e-30)
        assert dR[0, 0] == pytest.approx(4 * a * gv * (a * gv * gv - 1), rel=1e-13, abs=1e-15)


def test_rhs_residual_vanishes_at_the_exact_inverse_factor():
    """With G the inverse of the Cholesky factor of A (a full lower pattern),
    G^T G = A^{-1}: R = 0 and its gradient vanishes."""
    from types import SimpleNamespace
    rng = np.random.default_rng(8)
    M = rng.standard_normal((7, 7))
    A = M @ M.T + 7 * np.eye(7)
    G = np.linalg.inv(np.linalg.cholesky(A))
    R, dR = F.rhs_residual(SimpleNamespace(A=sp.csr_matrix(A)), sp.csr_matrix(np.tril(G)),
                           rng.standard_normal((7, 3)))
    assert R < 1e-28
    assert np.max(np.abs(dR.toarray())) < 1e-12


def test_rhs_residual_gradient_matches_finite_differences():
    g = _tiny_graph(5, 6)
    rng = np.random.default_rng(9)
    G = F.classical_fsai(g.A)
    G.data = G.data * (1 + 0.2 * rng.standard_normal(G.data.shape))
    B = rng.standard_normal((g.n, 3)) + 2.0
    R, dR = F.rhs_residual(g, G, B)
    Gc = G.tocoo()
    for t in rng.choice(Gc.nnz, 15, replace=False):
        i, j = Gc.row[t], Gc.col[t]
        h = 1e-6 * max(abs(Gc.data[t]), 1e-3)
        Gp = G.tolil(); Gp[i, j] += h
        Gm = G.tolil(); Gm[i, j] -= h
        fd = (F.rhs_residual(g, Gp.tocsr(), B)[0] - F.rhs_residual(g, Gm.tocsr(), B)[0]) / (2 * h)
        assert fd == pytest.approx(dR[i, j], rel=1e-5, abs=1e-10)


def test_network_gradient_with_the_rhs_term_matches_finite_differences():
    g = _tiny_graph(6, 5)
    rng = np.random.default_rng(10)
    th = F.init_params(7) + 0.05 * rng.standard_normal(F.NPARAM)
    B = rng.standard_normal((g.n, 2))
    L0 = F.loss_and_grad(th, g)[0]
    L, grad, info = F.loss_and_grad(th, g, B=B, mu=0.7)
    assert L == pytest.approx(L0 + 0.7 * info["R"], rel=1e-14)
    for k in rng.choice(F.NPARAM, 20, replace=False):
        h = 1e-6
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        fd = (F.loss_and_grad(tp, g, B=B, mu=0.7)[0] - F.loss_and_grad(tm, g, B=B, mu=0.7)[0]) / (2 * h)
        assert fd == pytest.approx(grad[k], rel=1e-5, abs=1e-9), k
