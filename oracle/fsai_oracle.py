"""FP64 oracle of the learned factorised-sparse-approximate-inverse (FSAI)
preconditioner for the PCG solve of Eq. 13.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg).  The paper
preconditions its conjugate gradients with incomplete Cholesky (Sec. III);
this learned preconditioner has no counterpart in the paper.  It is
M^{-1} = G^T G with G lower triangular on the pattern of tril(A):

* G = Gh diag(A)^{-1/2}: G_ij = Gh_ij / sqrt(A_jj); an untrained network
  (Gh = I) is exactly the Jacobi preconditioner.
* Gh_ii = softplus(h_diag), Gh_ij = h_off (j < i), from a 4 -> 64 -> 64 -> 2
  ReLU MLP evaluated once per pattern entry (n diagonal entries and one per
  undirected edge).
* Inputs of entry (b, a), a < b (edge e = (a, b), value G_ba):
  (rho_ab, theta_b, theta_a, w_ab) with rho_ab = lam w_ab^2 / sqrt(A_aa A_bb)
  (the Jacobi-scaled coupling), theta_i = r d_i / A_ii (the share of the
  constraint term in the diagonal) and the heat-kernel weight w_ab (a
  function of |x_a - x_b|).  Diagonal entry i: (s_i, theta_i, theta_i, 1)
  with s_i = sum over i's lower neighbours j of rho_ij^2.
* Training criterion: Kaporin's condition number of G A G^T,
      L = log(tr(G A G^T) / n) - (2/n) sum_i log G_ii   (+ log det A / n, constant),
  which classical FSAI minimises over the same pattern, optionally plus
  mu times the mean relative residual of the preconditioner on right-hand
  sides b_c the method itself produced (Eq. 13's right-hand sides),
      R = (1/m) sum_c |A G^T G b_c - b_c|^2 / |b_c|^2  (``rhs_residual``).

Training takes Adam steps (Kingma and Ba, ICLR 2015, Algorithm 1) on the
loss averaged over a mini-batch of images: ``adam_step``.

Parameter vector layout (float64 here, float32 on the GPU):
  W1 (4 x 64, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (64 x 2), b3 (2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

H = 64
NPARAM = 4 * H + H + H * H + H + H * 2 + 2
SOFTPLUS_ONE = float(np.log(np.expm1(1.0)))  # softplus^{-1}(1)


def unpack(theta: np.ndarray):
    o = 0
    W1 = theta[o:o + 4 * H].reshape(4, H); o += 4 * H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + 2 * H].reshape(H, 2); o += 2 * H
    b3 = theta[o:o + 2]; o += 2
    assert o == NPARAM
    return W1, b1, W2, b2, W3, b3


def init_params(seed: int = 0) -> np.ndarray:
    """He-initialised hidden layers, zero output layer, diagonal bias so that
    softplus(b3[1]) = 1: the untrained network gives Gh = I (Jacobi)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((4, H)) * np.sqrt(2.0 / 4)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    parts = [W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), np.zeros(2 * H), np.array([0.0, SOFTPLUS_ONE])]
    return np.concatenate(parts)


def softplus(x):
    return np.logaddexp(0.0, x)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def bf16_round(x):
    """Round to the nearest bfloat16 (8 significant bits, ties to even), via
    FP32: the rounding the GPU's tensor-core layer applies to its operands.
    Returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_forward(theta, F, bf16: bool = False):
    """out = ReLU(ReLU(F W1 + b1) W2 + b2) W3 + b3.  bf16: the 64 x 64 layer's
    operands (h1 and W2) rounded to bfloat16 first, as the GPU's tensor cores
    take them (everything else in FP64)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    a1 = F @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    if bf16:
        h1 = bf16_round(h1)
        W2 = bf16_round(W2)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    out = h2 @ W3 + b3
    return out, (F, a1, h1, a2, h2)


def mlp_backward(theta, cache, dout, bf16: bool = False):
    """Gradient of sum(out * dout) w.r.t. theta, back through mlp_forward's
    cache.  bf16: the 64 x 64 layer's backward products take bfloat16
    operands (da2, and W2 for dh1 = da2 W2^T; h1 is already rounded), as the
    GPU's tensor cores do."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    F, a1, h1, a2, h2 = cache
    gW3 = h2.T @ dout
    gb3 = dout.sum(0)
    dh2 = dout @ W3.T
    da2 = dh2 * (a2 > 0)
    gb2 = da2.sum(0)
    if bf16:
        da2 = bf16_round(da2)
        W2 = bf16_round(W2)
    gW2 = h1.T @ da2
    dh1 = da2 @ W2.T
    da1 = dh1 * (a1 > 0)
    gW1 = F.T @ da1
    gb1 = da1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def entry_features(g):
    """Features of the n diagonal entries and |E| edge entries of graph g
    (an oracle Graph: a < b edge lists, w, degrees, lambda, r, A)."""
    Ad = g.A.diagonal()
    theta = g.r * g.dvec / Ad
    rho = g.lam * g.w ** 2 / np.sqrt(Ad[g.a] * Ad[g.b])
    s = np.zeros(g.n)
    np.add.at(s, g.b, rho ** 2)                  # lower neighbours of row b are the a's
    Fd = np.stack([s, theta, theta, np.ones(g.n)], axis=1)
    Fe = np.stack([rho, theta[g.b], theta[g.a], g.w], axis=1)
    return Fd, Fe


def assemble_G(g, out_d, out_e):
    """G (sparse lower triangular) from the two heads."""
    Ad = g.A.diagonal()
    gd = softplus(out_d[:, 1]) / np.sqrt(Ad)
    ge = out_e[:, 0] / np.sqrt(Ad[g.a])          # G_ba, column a
    rows = np.concatenate([np.arange(g.n), g.b])
    cols = np.concatenate([np.arange(g.n), g.a])
    return sp.csr_matrix((np.concatenate([gd, ge]), (rows, cols)), shape=(g.n, g.n)), gd, ge


def kaporin(g, G):
    """L = log(tr(G A G^T)/n) - (2/n) sum log G_ii and dL/dG on G's pattern."""
    n = g.n
    GA = (G @ g.A).tocsr()
    T = float(G.multiply(GA).sum())
    gdiag = G.diagonal()
    L = np.log(T / n) - 2.0 / n * np.sum(np.log(gdiag))
    # dT/dG = 2 G A (restricted to the pattern); d(sum log G_ii)/dG_ii = 1/G_ii
    dG = (2.0 / T) * GA.multiply(G != 0).tocsr()
    dG = dG + sp.diags(-2.0 / (n * gdiag))
    return L, dG, T


def rhs_residual(g, G, B):
    """R = (1/m) sum_c |A G^T G b_c - b_c|^2 / |b_c|^2 over the m columns of
    B (n x m) and dR/dG on G's pattern (lower triangle with the diagonal).
    With u = G b, v = G^T u, w = A v - b and s = dR/dv = 2 A w / (m |b|^2)
    (A symmetric): v_j = sum_i G_ij u_i gives dR/dG_ij = u_i s_j, and u_i =
    sum_j G_ij b_j gives dR/dG_ij = (G s)_i b_j; both are kept where G has
    an entry."""
    m = B.shape[1]
    A = g.A.tocsr()
    bn = np.sum(B * B, axis=0)
    U = G @ B
    V = G.T @ U
    Wr = A @ V - B
    R = float(np.sum(np.sum(Wr * Wr, axis=0) / bn) / m)
    S = (A @ Wr) * (2.0 / (m * bn))
    GS = G @ S
    Gc = G.tocoo()
    i, j = Gc.row, Gc.col
    vals = np.sum(U[i] * S[j] + GS[i] * B[j], axis=1)
    return R, sp.csr_matrix((vals, (i, j)), shape=G.shape)


def loss_and_grad(theta, g, bf16: bool = False, B=None, mu: float = 0.0):
    """Kaporin loss of the network's G on graph g and its gradient w.r.t.
    theta (bf16: the hidden layer's operands rounded as on the GPU); with
    right-hand sides B (n x m) and mu > 0, plus mu times rhs_residual."""
    Fd, Fe = entry_features(g)
    od, cd = mlp_forward(theta, Fd, bf16)
    oe, ce = mlp_forward(theta, Fe, bf16)
    G, gd, ge = assemble_G(g, od, oe)
    L, dG, T = kaporin(g, G)
    Rr = None
    if B is not None and mu > 0.0:
        Rr, dR = rhs_residual(g, G, B)
        L = L + mu * Rr
        dG = dG.tocsr() + mu * dR
    Ad = g.A.diagonal()
    dG = dG.tocsr()
    dgd = np.asarray(dG[np.arange(g.n), np.arange(g.n)]).ravel()
    dge = np.asarray(dG[g.b, g.a]).ravel()
    dout_d = np.zeros_like(od)
    dout_d[:, 1] = dgd * sigmoid(od[:, 1]) / np.sqrt(Ad)
    dout_e = np.zeros_like(oe)
    dout_e[:, 0] = dge / np.sqrt(Ad[g.a])
    grad = mlp_backward(theta, cd, dout_d, bf16) + mlp_backward(theta, ce, dout_e, bf16)
    return L, grad, {"T": T, "gd": gd, "ge": ge, "G": G, "R": Rr}


def classical_fsai(A) -> sp.csr_matrix:
    """Classical FSAI on the pattern of tril(A): for row i with pattern S
    (i last), solve A[S, S] g = e_i and scale by 1/sqrt(g_i).  Minimises the
    Kaporin number of G A G^T over lower-triangular G with that pattern."""
    A = A.tocsr()
    n = A.shape[0]
    Lp = sp.tril(A).tocsr()
    rows, cols, vals = [], [], []
    for i in range(n):
        S = np.sort(Lp.indices[Lp.indptr[i]:Lp.indptr[i + 1]])
        As = A[S][:, S].toarray()
        e = np.zeros(len(S))
        e[-1] = 1.0
        gi = np.linalg.solve(As, e)
        gi = gi / np.sqrt(gi[-1])
        rows += [i] * len(S)
        cols += list(S)
        vals += list(gi)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def fsai_apply(G, R):
    """z = G^T (G r), column by column."""
    return G.T @ (G @ R)


def adam_step(theta, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One step of Adam (Kingma and Ba, ICLR 2015, Algorithm 1), the
    optimiser of the network's training: exponential moving averages of the
    gradient and of its square, each divided by its bias correction
    1 - beta^step, and a step of lr * mhat / (sqrt(vhat) + eps).
    Returns (theta, m, v) after the step; the inputs are not changed."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
