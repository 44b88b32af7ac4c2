"""FP64 CPU oracle for piecewise flat embeddings (PFE).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  The CUDA
library never calls it and shares no code with it.

It follows the paper (Meinhold, Hayes & Cahill, "Efficiently Computing
Piecewise Flat Embeddings for Data Clustering and Image Segmentation"):

* Sec. II, heat kernel: w_ij = exp(-|x_i - x_j|^2 / (2 sigma^2)).
* Sec. II, degree matrix: D = diag(d), d_i = sum_j w_ij.
* Sec. II, edge operator M: one row per undirected edge (i, j), with +w_ij in
  column i and -w_ij in column j.
* Alg. 1 (SOC): P = D^{1/2} Y, B = 0; repeat {Y-step; P-step; B-step}.
* Alg. 2 (split Bregman) with the compact substitutions of Eqs. 9, 10 and 13:
  the normal equations [lam M^T M + r D] Y = lam M^T Q1 + r D^{1/2} Q2 are d
  independent n x n systems sharing one matrix.
* Alg. 2, Shrink: z = sign(y) * max(|y| - gamma, 0).
* Sec. III (end): the solve is done by preconditioned conjugate gradients.
  Here the parity mode solves it exactly (sparse LU, factored once because
  the matrix is constant) and the timing mode runs Jacobi-preconditioned CG.

Readings where the paper is silent or garbled (each is listed in the design
notes of the repository):

* Q2 = P - B.  Eq. 6 and Eq. 13 print Q2 = B - P, but setting the gradient of
  Alg. 2 step 5's objective to zero gives r D^{1/2}(P - B) on the right.
* Alg. 1 step 5 prints "D^{1/2}Y - P + P"; the second P is read as B, as in
  Eq. 5 and the B-step.
* The P-step's closed form is not printed (it is deferred to Yu et al.); it is
  the orthogonal Procrustes minimiser, i.e. the polar factor U V^T of
  X = D^{1/2}Y + B = U S V^T.
* The edge set is the undirected pairs (i < j) with nonzero weight, so
  M^T M = D2 - W.W (the Laplacian of the squared weights), D2 = diag(sum_j w_ij^2).
* The inner state (b, d) restarts at zero on every call of Alg. 2.
* lam defaults to sqrt(vol) = sqrt(sum_i d_i), r to 1 (values are not printed).
* The starting embedding is D-orthonormalised by the same polar step:
  Y0 <- D^{-1/2} polar(D^{1/2} Y0).
* The Laplacian-eigenmap start (Sec. I) is the d smallest generalised
  eigenvectors of (D - W) v = mu D v on the D-orthogonal complement of the
  constant vector, D-normalised, each with its largest-magnitude entry made
  positive (ties: the smallest index).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# --------------------------------------------------------------------------
# Graph (Sec. II and Sec. IV)
# --------------------------------------------------------------------------


def grid_offsets(radius: float) -> list[tuple[int, int]]:
    """All pixel offsets (dx, dy) with 0 < dx^2 + dy^2 <= radius^2 (Sec. IV)."""
    R = int(np.floor(radius))
    out = []
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            if 0 < dx * dx + dy * dy <= radius * radius:
                out.append((dx, dy))
    return out


def grid_edges(H: int, W: int, radius: float) -> tuple[np.ndarray, np.ndarray]:
    """Undirected edges (a, b), a < b, between pixels within ``radius``.

    Pixel (x, y) is vertex y*W + x.  Each unordered pair is listed once; the
    list is sorted by (a, b).
    """
    aa, bb = [], []
    ys, xs = np.mgrid[0:H, 0:W]
    p = ys * W + xs
    for dx, dy in grid_offsets(radius):
        x2, y2 = xs + dx, ys + dy
        ok = (x2 >= 0) & (x2 < W) & (y2 >= 0) & (y2 < H)
        a = p[ok]
        b = (y2 * W + x2)[ok]
        keep = a < b
        aa.append(a[keep])
        bb.append(b[keep])
    a = np.concatenate(aa)
    b = np.concatenate(bb)
    order = np.lexsort((b, a))
    return a[order].astype(np.int64), b[order].astype(np.int64)


def heat_kernel_weights(X: np.ndarray, a: np.ndarray, b: np.ndarray, sigma: float) -> np.ndarray:
    """w_ab = exp(-|x_a - x_b|^2 / (2 sigma^2)) (Sec. II, heat kernel)."""
    diff = X[a] - X[b]
    return np.exp(-np.sum(diff * diff, axis=1) / (2.0 * sigma * sigma))


def adjacency(n: int, a: np.ndarray, b: np.ndarray, w: np.ndarray) -> sp.csr_matrix:
    """Symmetric weighted adjacency W (Sec. II)."""
    Wm = sp.coo_matrix((np.concatenate([w, w]), (np.concatenate([a, b]), np.concatenate([b, a]))),
                       shape=(n, n))
    return Wm.tocsr()


def degrees(Wm: sp.csr_matrix) -> np.ndarray:
    """d = W 1 (Sec. II; Alg. 1 step 2)."""
    return np.asarray(Wm.sum(axis=1)).ravel()


def edge_operator(n: int, a: np.ndarray, b: np.ndarray, w: np.ndarray) -> sp.csr_matrix:
    """M: row e has +w_e in column a_e and -w_e in column b_e (Sec. II)."""
    E = a.shape[0]
    rows = np.concatenate([np.arange(E), np.arange(E)])
    cols = np.concatenate([a, b])
    vals = np.concatenate([w, -w])
    return sp.csr_matrix((vals, (rows, cols)), shape=(E, n))


def default_lambda(dvec: np.ndarray) -> float:
    """lam = sqrt(vol(W)) (reading; the paper defers the value to Yu et al.)."""
    return float(np.sqrt(np.sum(dvec)))


def system_matrix(M: sp.csr_matrix, dvec: np.ndarray, lam: float, r: float) -> sp.csr_matrix:
    """A = lam M^T M + r D, Eq. 13's left side times 2."""
    return (lam * (M.T @ M) + r * sp.diags(dvec)).tocsr()


@dataclass
class Graph:
    """Everything the iteration needs about one data set."""

    n: int
    a: np.ndarray
    b: np.ndarray
    w: np.ndarray
    dvec: np.ndarray
    M: sp.csr_matrix
    lam: float
    r: float
    A: sp.csr_matrix

    @property
    def n_edges(self) -> int:
        return int(self.a.shape[0])


def build_graph(X: np.ndarray, a: np.ndarray, b: np.ndarray, sigma: float,
                lam: float | None = None, r: float = 1.0) -> Graph:
    """Heat-kernel graph, degrees, edge operator and system matrix."""
    n = X.shape[0]
    w = heat_kernel_weights(X, a, b, sigma)
    Wm = adjacency(n, a, b, w)
    dvec = degrees(Wm)
    if np.any(dvec <= 0):
        raise ValueError("a vertex has zero degree; D^{-1/2} is undefined")
    M = edge_operator(n, a, b, w)
    if lam is None or lam <= 0:
        lam = default_lambda(dvec)
    A = system_matrix(M, dvec, lam, r)
    return Graph(n, a, b, w, dvec, M, float(lam), float(r), A)


def build_grid_graph(X: np.ndarray, H: int, W: int, radius: float, sigma: float,
                     lam: float | None = None, r: float = 1.0) -> Graph:
    a, b = grid_edges(H, W, radius)
    return build_graph(X, a, b, sigma, lam, r)


# --------------------------------------------------------------------------
# Pointwise pieces
# --------------------------------------------------------------------------


def shrink(y: np.ndarray, gamma: float) -> np.ndarray:
    """Alg. 2, Shrink: sign(y) * max(|y| - gamma, 0), elementwise."""
    return np.sign(y) * np.maximum(np.abs(y) - gamma, 0.0)


def polar_factor(X: np.ndarray) -> np.ndarray:
    """argmin_P |P - X|_F s.t. P^T P = I: U V^T from the thin SVD X = U S V^T.

    Alg. 1 step 6 (closed form read as the orthogonal Procrustes solution).
    Raises when X is rank deficient, where the minimiser is not unique.
    """
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    if s.size == 0 or s[-1] <= 1e-14 * s[0]:
        raise np.linalg.LinAlgError("P-step: X is numerically rank deficient")
    return U @ Vt


def d_orthonormalize(Y0: np.ndarray, dvec: np.ndarray) -> np.ndarray:
    """Y = D^{-1/2} polar(D^{1/2} Y0), so that Y^T D Y = I (Eq. 1 constraint)."""
    sq = np.sqrt(dvec)[:, None]
    return polar_factor(sq * Y0) / sq


def sign_fix(V: np.ndarray) -> np.ndarray:
    """Deterministic sign of each column: the entry of largest magnitude is
    made positive (ties: the smallest row index)."""
    V = np.array(V, dtype=np.float64, copy=True)
    for c in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, c])))  # argmax returns the first maximum
        if V[i, c] < 0:
            V[:, c] = -V[:, c]
    return V


def laplacian_eigenmap(g: Graph, d: int) -> np.ndarray:
    """Laplacian-eigenmap start (Sec. I; Belkin & Niyogi): the generalised
    eigenvectors of (D - W) v = mu D v for the d smallest mu on the
    D-orthogonal complement of the constant vector (the trivial solution,
    mu = 0), in ascending mu, each with v^T D v = 1 and its sign fixed by
    ``sign_fix``.  On a connected graph this drops the first eigenvector; on
    a graph of k components it keeps the k - 1 piecewise-constant directions
    orthogonal to the constant one.

    The d + 1 smallest eigenvectors come from dense ``scipy.linalg.eigh``
    (n <= 3000) or shift-invert Lanczos (``scipy.sparse.linalg.eigsh``);
    the constant direction is then removed inside their span and the rest
    rotated back to eigenvectors (Rayleigh-Ritz)."""
    Wm = adjacency(g.n, g.a, g.b, g.w)
    Dm = sp.diags(g.dvec)
    L = (Dm - Wm).tocsc()
    if g.n <= 3000:
        import scipy.linalg as sla
        mu, V = sla.eigh(L.toarray(), np.diag(g.dvec), subset_by_index=[0, d])
    else:
        shift = -1e-6 * float(np.max(g.dvec))
        mu, V = spla.eigsh(L, k=d + 1, M=Dm.tocsc(), sigma=shift, which="LM")
        order = np.argsort(mu)
        mu, V = mu[order], V[:, order]
    V = V / np.sqrt(np.einsum("ic,i,ic->c", V, g.dvec, V))[None, :]
    # coordinates of the D-unit constant vector in the (D-orthonormal) basis V,
    # and an orthonormal basis of their complement in R^{d+1}
    vol = float(np.sum(g.dvec))
    cvec = V.T @ g.dvec / np.sqrt(vol)
    _, _, Vt = np.linalg.svd(cvec[None, :])
    Vp = V @ Vt[1:].T                        # D-orthonormal, D-orthogonal to the constant
    H = Vp.T @ (L @ Vp)
    theta, C = np.linalg.eigh(0.5 * (H + H.T))
    Vp = Vp @ C                               # ascending Rayleigh quotients
    Vp = Vp / np.sqrt(np.einsum("ic,i,ic->c", Vp, g.dvec, Vp))[None, :]
    return sign_fix(Vp)


def objective(g: Graph, Y: np.ndarray) -> float:
    """|M Y|_1 = sum over undirected edges of w_ab |y_a - y_b|_1 (Eq. 1 counts each pair twice)."""
    return float(np.abs(g.M @ Y).sum())


# --------------------------------------------------------------------------
# Linear solves of Eq. 13
# --------------------------------------------------------------------------


class DirectSolver:
    """Exact solve of A Y = RHS; A is factored once (it is constant over the run)."""

    def __init__(self, A: sp.csr_matrix):
        self.lu = spla.splu(A.tocsc())

    def __call__(self, rhs: np.ndarray, y0: np.ndarray | None = None):
        Y = self.lu.solve(np.asarray(rhs, dtype=np.float64))
        d = rhs.shape[1]
        return Y, {"iters": np.zeros(d, dtype=np.int64), "relres": np.zeros(d)}


def jacobi_pcg(A: sp.csr_matrix, Bm: np.ndarray, X0: np.ndarray, tol: float, max_iter: int,
               refresh: int = 50):
    """d independent Jacobi-preconditioned CG runs on A x_c = b_c (Sec. III).

    The textbook PCG recurrences (Barrett et al., Templates, Fig. 2.5) run on
    every column with its own alpha and beta.  A column stops once
    |b_c - A x_c| / |b_c| <= tol (it is then left unchanged); every
    ``refresh`` iterations the recursive residual is replaced by b - A x.
    Returns (X, info) with per-column iteration counts and relative residuals.
    """
    diag_inv = 1.0 / A.diagonal()
    return pcg(A, Bm, X0, tol, max_iter, refresh, lambda R: diag_inv[:, None] * R)


def pcg(A: sp.csr_matrix, Bm: np.ndarray, X0: np.ndarray, tol: float, max_iter: int,
        refresh: int, apply_minv):
    """The PCG runs of ``jacobi_pcg`` with any preconditioner: apply_minv(R)
    returns Z = M^{-1} R column by column (for an FSAI factor G, G^T G R)."""
    X = np.array(X0, dtype=np.float64, copy=True)
    Bm = np.asarray(Bm, dtype=np.float64)
    d = Bm.shape[1]
    bnorm = np.linalg.norm(Bm, axis=0)
    bnorm_safe = np.where(bnorm > 0, bnorm, 1.0)
    R = Bm - A @ X
    iters = np.zeros(d, dtype=np.int64)
    relres = np.linalg.norm(R, axis=0) / bnorm_safe
    active = relres > tol
    Z = apply_minv(R)
    P = Z.copy()
    rz = np.sum(R * Z, axis=0)
    k = 0
    while np.any(active) and k < max_iter:
        Q = A @ P
        pq = np.sum(P * Q, axis=0)
        alpha = np.where(active, rz / np.where(pq != 0, pq, 1.0), 0.0)
        X += alpha[None, :] * P
        R -= alpha[None, :] * Q
        k += 1
        iters[active] = k
        if refresh > 0 and k % refresh == 0:
            R = np.where(active[None, :], Bm - A @ X, R)
        Z = apply_minv(R)
        rz_new = np.sum(R * Z, axis=0)
        relres = np.linalg.norm(R, axis=0) / bnorm_safe
        now_done = active & (relres <= tol)
        active = active & ~now_done
        beta = np.where(active, rz_new / np.where(rz != 0, rz, 1.0), 0.0)
        P = Z + beta[None, :] * P
        rz = rz_new
    true_rel = np.linalg.norm(Bm - A @ X, axis=0) / bnorm_safe
    return X, {"iters": iters, "relres": relres, "true_relres": true_rel,
               "converged": bool(not np.any(active))}


class PCGSolver:
    def __init__(self, A: sp.csr_matrix, tol: float, max_iter: int = 5000, refresh: int = 50):
        self.A, self.tol, self.max_iter, self.refresh = A, tol, max_iter, refresh

    def __call__(self, rhs: np.ndarray, y0: np.ndarray):
        return jacobi_pcg(self.A, rhs, y0, self.tol, self.max_iter, self.refresh)


# --------------------------------------------------------------------------
# Alg. 2 and Alg. 1
# --------------------------------------------------------------------------


@dataclass
class State:
    """Iteration state of Alg. 1 / Alg. 2 (paper names in comments)."""

    Y: np.ndarray          # current Y (last split-Bregman solve)
    P: np.ndarray          # P^(k)
    B: np.ndarray          # B^(k)
    bs: np.ndarray         # b^l, one row per undirected edge
    ds: np.ndarray         # d^l, one row per undirected edge
    outer: int = 0
    inner: int = 0
    history: list = field(default_factory=list)


def init_state(g: Graph, Y0: np.ndarray) -> State:
    """Alg. 1 step 3 after D-orthonormalising the starting embedding."""
    Y = d_orthonormalize(Y0, g.dvec)
    P = np.sqrt(g.dvec)[:, None] * Y
    B = np.zeros_like(P)
    z = np.zeros((g.n_edges, Y.shape[1]))
    return State(Y=Y, P=P, B=B, bs=z.copy(), ds=z.copy())


def split_bregman_step(g: Graph, st: State, solve) -> dict:
    """One pass of Alg. 2 steps 5-7 in the compact form (Eqs. 13, 9, 10)."""
    sq = np.sqrt(g.dvec)[:, None]
    Q1 = st.ds - st.bs                      # d^l - b^l
    Q2 = st.P - st.B                        # reading: P - B
    rhs = g.lam * (g.M.T @ Q1) + g.r * sq * Q2
    Y, info = solve(rhs, st.Y)              # Eq. 13
    MY = g.M @ Y                            # Eq. 7
    ds = shrink(MY + st.bs, 1.0 / g.lam)    # Eq. 9
    bs = st.bs + MY - ds                    # Eq. 10
    st.Y, st.ds, st.bs = Y, ds, bs
    st.inner += 1
    return info


def p_and_b_step(g: Graph, st: State) -> None:
    """Alg. 1 steps 6-7: P = polar(D^{1/2}Y + B); B = B + D^{1/2}Y - P."""
    sq = np.sqrt(g.dvec)[:, None]
    Xm = sq * st.Y + st.B
    P = polar_factor(Xm)
    st.B = st.B + sq * st.Y - P
    st.P = P
    st.outer += 1


def reset_inner(st: State) -> None:
    """Alg. 2 step 3: b = d = 0 at the start of every call."""
    st.bs[:] = 0.0
    st.ds[:] = 0.0


def soc_pfe(g: Graph, Y0: np.ndarray, n_outer: int, n_inner: int, solver: str = "direct",
            tol: float = 1e-8, max_iter: int = 5000, refresh: int = 50,
            reset_each_outer: bool = True, record: bool = False) -> State:
    """Alg. 1 with Alg. 2 as its Y-step, fixed iteration counts.

    Returns the final state; ``state.Y`` is the last split-Bregman solution and
    D^{-1/2} state.P (see ``embedding``) satisfies Y^T D Y = I.
    """
    st = init_state(g, Y0)
    solve = DirectSolver(g.A) if solver == "direct" else PCGSolver(g.A, tol, max_iter, refresh)
    for _ in range(n_outer):
        if reset_each_outer or st.outer == 0:
            reset_inner(st)
        for _ in range(n_inner):
            info = split_bregman_step(g, st, solve)
            if record:
                st.history.append({"outer": st.outer, "iters": info["iters"].copy(),
                                   "relres": np.array(info["relres"]).copy()})
        p_and_b_step(g, st)
    return st


def two_stage(g: Graph, Y0: np.ndarray, n_outer: int, n_inner: int, n_stage2: int, solver: str = "direct",
              tol: float = 1e-8, max_iter: int = 5000, refresh: int = 50) -> State:
    """Sec. IV two-stage schedule.  Stage I: Alg. 1 (n_outer SOC iterations
    of n_inner split-Bregman iterations each).  Stage II: the orthogonality
    constraint is relaxed -- P and B keep their Stage I values, so it is only
    penalised by the r-term -- and one more call of Alg. 2 (b = d = 0 at its
    start) runs n_stage2 split-Bregman iterations.  ``state.Y`` is Stage
    II's Y; P, B (and ``embedding``) are Stage I's."""
    st = soc_pfe(g, Y0, n_outer, n_inner, solver, tol, max_iter, refresh)
    solve = DirectSolver(g.A) if solver == "direct" else PCGSolver(g.A, tol, max_iter, refresh)
    reset_inner(st)
    for _ in range(n_stage2):
        split_bregman_step(g, st, solve)
    return st


def embedding(g: Graph, st: State) -> np.ndarray:
    """Yhat = D^{-1/2} P, the D-orthonormal embedding."""
    return st.P / np.sqrt(g.dvec)[:, None]
