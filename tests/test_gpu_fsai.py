"""Learned FSAI preconditioner on the GPU (through the C ABI) against the
FP64 oracle.  The hidden layer runs with BF16 operands, so network outputs
carry ~2^-9 relative rounding; tolerances below are set from that."""
import numpy as np
import pytest

from oracle import fsai_oracle as F
from oracle import pfe_oracle as O
from synth import make_problem
from tests.gpu_common import gpu_problem, oracle_graph, relerr, small_spec

pytestmark = pytest.mark.gpu


def _perturbed_params(seed=3, scale=0.05):
    th = F.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    return th + scale * rng.standard_normal(th.shape)


def test_untrained_network_is_jacobi():
    spec = small_spec(H=17, W=19, d=3)
    p, X, Y0 = gpu_problem(spec, "mixed")
    g = oracle_graph(spec, X)
    p.fsai_set(F.init_params(0).astype(np.float32))
    gd, ge = p.fsai_get()
    np.testing.assert_allclose(gd, 1.0 / np.sqrt(g.A.diagonal()), rtol=2e-6)
    assert np.all(ge == 0.0)
    p.close()


def test_fsai_forward_matches_oracle():
    """G from the GPU's network against the oracle's network with the hidden
    layer's operands rounded to BF16 as on the tensor cores (what is left is
    FP32 features and accumulation: 1e-4), and within the BF16 rounding of
    the FP64 network."""
    spec = small_spec(H=21, W=23, d=3, radius=3.0)
    p, X, Y0 = gpu_problem(spec, "mixed")
    g = oracle_graph(spec, X)
    th = _perturbed_params()
    p.fsai_set(th.astype(np.float32))
    gd, ge = p.fsai_get()
    th32 = th.astype(np.float32).astype(np.float64)  # the parameters the GPU holds
    Fd, Fe = F.entry_features(g)
    for bf16, bd, be in ((True, 1e-4, 1e-4), (False, 1e-2, 3e-2)):
        od, _ = F.mlp_forward(th32, Fd, bf16)
        oe, _ = F.mlp_forward(th32, Fe, bf16)
        _, gd_ref, ge_ref = F.assemble_G(g, od, oe)
        assert relerr(gd, gd_ref) < bd, (bf16, relerr(gd, gd_ref))
        assert relerr(ge, ge_ref) < be, (bf16, relerr(ge, ge_ref))
    p.close()


@pytest.mark.parametrize("H,W,d,radius", [(12, 13, 2, 2.0), (23, 19, 3, 3.0)])
def test_fsai_loss_and_gradient_match_oracle(H, W, d, radius):
    """Kaporin loss and its gradient through the GPU's forward and backward
    kernels against the oracle with the same BF16 roundings of the hidden
    layer's operands (h1, W2 and the backward's da2): relative error <= 1e-3
    (what remains is FP32 accumulation and FP32 features), on two images."""
    spec = small_spec(H=H, W=W, d=d, radius=radius)
    p, X, Y0 = gpu_problem(spec, "mixed")
    g = oracle_graph(spec, X)
    th = _perturbed_params(5, 0.05).astype(np.float32)
    th64 = th.astype(np.float64)
    L_ref, grad_ref, _ = F.loss_and_grad(th64, g, bf16=True)
    L, grad = p.fsai_loss_grad(th)
    assert abs(L - L_ref) <= 1e-5 * max(1.0, abs(L_ref)), (L, L_ref)
    assert relerr(grad, grad_ref) <= 1e-3, relerr(grad, grad_ref)
    # and the FP64 network's gradient is within the BF16 rounding of it
    _, grad64, _ = F.loss_and_grad(th64, g)
    assert relerr(grad, grad64) < 0.1
    p.close()


def test_pcg_with_fsai_solves_exactly():
    spec = small_spec(H=26, W=24, d=4)
    p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-6)
    g = oracle_graph(spec, X)
    p.init(Y0)
    p.fsai_set(_perturbed_params(7, 0.02).astype(np.float32))
    rng = np.random.default_rng(9)
    R = rng.standard_normal((g.n, 4))
    Y = np.zeros_like(R)
    st = p.solve_system(R, Y)
    assert st["converged"]
    assert relerr(Y, O.DirectSolver(g.A)(R)[0]) < 1e-4
    # and the whole iteration runs with it (graph loop)
    Yo = np.empty((spec.n, 4))
    s = p.solve(2, 3, Yo, None)
    assert s["n_unconverged"] == 0
    p.close()


def test_classical_fsai_matches_oracle_and_cuts_iterations():
    spec = small_spec(H=30, W=28, d=3, radius=3.0)
    p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-6)
    g = oracle_graph(spec, X)
    p.init(Y0)
    rng = np.random.default_rng(11)
    R = rng.standard_normal((g.n, 3))
    Y = np.zeros_like(R)
    it_jacobi = p.solve_system(R, Y)["pcg_iters"]
    p.fsai_classical()
    gd, ge = p.fsai_get()
    G = F.classical_fsai(g.A).tocsr()
    np.testing.assert_allclose(gd, G.diagonal(), rtol=1e-6)
    np.testing.assert_allclose(ge, np.asarray(G[g.b, g.a]).ravel(), rtol=1e-5, atol=1e-7 * np.abs(ge).max())
    Y = np.zeros_like(R)
    st = p.solve_system(R, Y)
    assert st["converged"] and st["pcg_iters"] < it_jacobi
    assert relerr(Y, O.DirectSolver(g.A)(R)[0]) < 1e-4
    p.close()


@pytest.mark.parametrize("radius", [2.0, 3.0])
def test_fsai_pcg_iterations_match_oracle(radius):
    """PCG with M^-1 = G^T G for the classical FSAI factor: the number of
    iterations the GPU needs to reach the tolerance (its r.z taken as |G r|^2)
    against the oracle's FP64 PCG with the same G (r.z taken directly), and
    the solutions.  Radius 2 and 3 run the fixed-row kernels of 12 and 28 slots."""
    spec = small_spec(H=31, W=29, d=3, radius=radius)
    p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-6)
    g = oracle_graph(spec, X)
    p.init(Y0)
    p.fsai_classical()
    G = F.classical_fsai(g.A).tocsr()
    rng = np.random.default_rng(23)
    R = rng.standard_normal((g.n, 3))
    Y = np.zeros_like(R)
    st = p.solve_system(R, Y)
    Yo, info = O.pcg(g.A, R, np.zeros_like(R), 1e-6, 5000, 50, lambda Rm: F.fsai_apply(G, Rm))
    assert st["converged"] and info["converged"]
    # FP32 vectors against FP64: the counts may differ by a step or two
    assert abs(st["pcg_iters"] - int(info["iters"].max())) <= 2, (st["pcg_iters"], info["iters"])
    assert relerr(Y, Yo) < 1e-4
    p.close()


def test_trained_network_cuts_pcg_iterations_on_the_gpu():
    """The committed weights through the GPU's BF16 tensor-core network and
    FSAI kernels: fewer PCG iterations than Jacobi on an image the network
    was not trained on (the oracle needs 0.54x), about as many as the oracle
    with the same weights, and the exact solution."""
    from paper_1612_06496_gb300.learned import load_weights
    spec = small_spec(H=40, W=48, d=4, seed=11, regions=4)
    p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-6)
    g = oracle_graph(spec, X)
    p.init(Y0)
    R = np.random.default_rng(31).standard_normal((g.n, 4))
    Yj = np.zeros_like(R)
    it_j = p.solve_system(R, Yj)["pcg_iters"]
    p.fsai_set(load_weights())
    Y = np.zeros_like(R)
    st = p.solve_system(R, Y)
    th = load_weights().astype(np.float64)
    Fd, Fe = F.entry_features(g)
    od, _ = F.mlp_forward(th, Fd)
    oe, _ = F.mlp_forward(th, Fe)
    G, _, _ = F.assemble_G(g, od, oe)
    _, info = O.pcg(g.A, R, np.zeros_like(R), 1e-6, 5000, 50, lambda Q: F.fsai_apply(G, Q))
    n_o = int(info["iters"].max())
    assert st["converged"] and st["pcg_iters"] <= 0.8 * it_j, (st["pcg_iters"], it_j)
    assert abs(st["pcg_iters"] - n_o) <= max(3, 0.25 * n_o), (st["pcg_iters"], n_o)
    assert relerr(Y, O.DirectSolver(g.A)(R)[0]) < 1e-4
    p.close()


def test_adam_kernel_matches_oracle():
    """pfe_adam_update (FP32, in place on device arrays) against the oracle's
    FP64 Adam step, on a length that is not a multiple of the block, at step
    3 from non-zero moments.  FP32 bounds: m from its two terms' sizes (they
    may cancel), v (non-negative terms) relative, the parameter to its own
    rounding plus the update's error at the scale of its terms."""
    import torch
    from paper_1612_06496_gb300.pfe import adam_update
    from tests.gpu_common import ensure_built
    ensure_built()
    rng = np.random.default_rng(9)
    # hyper-parameters that FP32 holds exactly, so both sides use the same
    # values (FP32 rounding of 0.999 alone would move 1 - b2 by 5e-5)
    n, step, lr, b1, b2, eps = 1000, 3, 2.0 ** -7, 0.875, 1 - 2.0 ** -10, 2.0 ** -27
    p0 = rng.standard_normal(n).astype(np.float32)
    g = (rng.standard_normal(n) * np.logspace(-3, 1, n)).astype(np.float32)
    m0 = (0.1 * rng.standard_normal(n)).astype(np.float32)
    v0 = rng.uniform(0.0, 1.0, n).astype(np.float32)
    P, G, M, V = (torch.from_numpy(a.copy()).cuda() for a in (p0, g, m0, v0))
    adam_update(P, G, M, V, step, lr, b1, b2, eps)
    torch.cuda.synchronize()
    f64 = [a.astype(np.float64) for a in (p0, g, m0, v0)]
    th, m, v = F.adam_step(*f64, step, lr, b1, b2, eps)
    u32 = 2.0 ** -23
    m_terms = np.abs(b1 * f64[2]) + np.abs((1 - b1) * f64[1])
    assert np.all(np.abs(M.cpu().numpy() - m) <= 4 * u32 * m_terms)
    np.testing.assert_allclose(V.cpu().numpy(), v, rtol=4 * u32)
    u_terms = lr * (m_terms / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    err = np.abs(P.cpu().numpy().astype(np.float64) - th)
    assert np.all(err <= u32 * np.abs(th) + 16 * u32 * u_terms)


@pytest.mark.parametrize("H,W,d,radius", [(12, 13, 2, 2.0), (23, 19, 3, 3.0)])
def test_fsai_rhs_term_matches_oracle(H, W, d, radius):
    """The training criterion with the right-hand-side term, mu times the
    mean of |A G^T G b - b|^2 / |b|^2 over a right-hand side of Eq. 13 that
    the method produced (after one inner step), through the GPU's forward,
    Kaporin and right-hand-side kernels and the network's backward, against
    the oracle with the same BF16 roundings: R to 1e-3, the loss to 1e-4,
    the gradient to 1e-3 (FP32 network output and accumulation); mu = 0
    gives the Kaporin loss and gradient bit for bit."""
    spec = small_spec(H=H, W=W, d=d, radius=radius)
    p, X, Y0 = gpu_problem(spec, "mixed")
    g = oracle_graph(spec, X)
    p.init(Y0)
    p.inner_step()
    B = np.ascontiguousarray(p.get("RHS"))
    th = _perturbed_params(5, 0.05).astype(np.float32)
    mu = 0.5
    L_ref, grad_ref, info = F.loss_and_grad(th.astype(np.float64), g, bf16=True, B=B, mu=mu)
    L, grad, R = p.fsai_loss_grad_rhs(th, B, mu)
    assert abs(R - info["R"]) <= 1e-3 * info["R"], (R, info["R"])
    assert abs(L - L_ref) <= 1e-4 * max(1.0, abs(L_ref)), (L, L_ref)
    assert relerr(grad, grad_ref) <= 1e-3, relerr(grad, grad_ref)
    L0, g0, R0 = p.fsai_loss_grad_rhs(th, B, 0.0)
    L1, g1 = p.fsai_loss_grad(th)
    assert L0 == L1 and R0 == 0.0
    np.testing.assert_array_equal(g0, g1)
    p.close()


@pytest.mark.parametrize("lam_scale,r", [(0.2, 1.0), (5.0, 1.0), (1.0, 4.0), (1.0, 0.25)])
def test_trained_network_away_from_its_training_lambda_and_r(lam_scale, r):
    """The network was trained with lambda = sqrt(vol W), r = 1.  Its inputs
    are scale-free quantities of A (the Jacobi-scaled coupling lam w^2 /
    sqrt(A_aa A_bb) and the share r d_i / A_ii of the constraint term), so
    other lambda and r change its inputs, not their meaning.  At lambda
    scaled by 0.2 and 5 and at r = 4 and 0.25 the learned factor still gives
    the oracle's solution of the whole nested loop (FP32 path, 2e-4) and
    still needs fewer PCG iterations than Jacobi, within 30 % of the
    classical FSAI (the pattern's Kaporin optimum)."""
    from paper_1612_06496_gb300.learned import load_weights
    spec = small_spec(H=48, W=52, d=4, seed=13, regions=4)
    X, Y0 = make_problem(spec)
    g0 = oracle_graph(spec, X)
    lam = lam_scale * g0.lam
    g = O.build_grid_graph(X, spec.H, spec.W, spec.radius, spec.sigma, lam=lam, r=r)
    ref = O.soc_pfe(g, Y0, 1, 3, solver="direct")
    its = {}
    for kind in ("jacobi", "classical", "learned"):
        p, _, _ = gpu_problem(spec, "mixed", tol=1e-6, lam=lam, r=r)
        p.init(Y0)
        if kind == "classical":
            p.fsai_classical()
        elif kind == "learned":
            p.fsai_set(load_weights())
        Y = np.empty_like(Y0)
        st = p.solve(1, 3, Y, None)
        assert st["n_unconverged"] == 0
        assert relerr(Y, ref.Y) <= 2e-4, (kind, relerr(Y, ref.Y))
        its[kind] = st["pcg_iters_total"]
        p.close()
    assert its["learned"] < its["jacobi"], its
    assert its["learned"] <= 1.3 * its["classical"], its


@pytest.mark.parametrize("H,W,d,radius", [(21, 23, 3, 3.0), (37, 41, 4, 2.0), (64, 64, 5, 2.0)])
def test_tcgen05_inference_matches_mma_sync_and_oracle(H, W, d, radius):
    """The learned factor's inference on the 5th-generation tensor cores
    (128 x 64 x 64 tcgen05.mma per 128 pattern entries, FP32 accumulator in
    tensor memory, the default) against the mma.sync form and the oracle:
    both take the same BF16 operands and accumulate in FP32 (in another
    order), so G agrees to 1e-5 between them, and to the oracle with the
    same BF16 roundings within 1e-4 (FP32 features and accumulation);
    entry counts that leave a ragged last tile of 128."""
    spec = small_spec(H=H, W=W, d=d, radius=radius)
    p, X, Y0 = gpu_problem(spec, "mixed")
    g = oracle_graph(spec, X)
    th = _perturbed_params().astype(np.float32)
    assert p.get_variant("mlp")[0] == 1
    p.fsai_set(th)
    gd1, ge1 = p.fsai_get()
    p.set_variant(0, "mlp")
    p.fsai_set(th)
    gd0, ge0 = p.fsai_get()
    assert relerr(gd1, gd0) < 1e-5 and relerr(ge1, ge0) < 1e-5, (relerr(gd1, gd0), relerr(ge1, ge0))
    Fd, Fe = F.entry_features(g)
    th32 = th.astype(np.float64)
    od, _ = F.mlp_forward(th32, Fd, True)
    oe, _ = F.mlp_forward(th32, Fe, True)
    _, gd_ref, ge_ref = F.assemble_G(g, od, oe)
    assert relerr(gd1, gd_ref) < 1e-4 and relerr(ge1, ge_ref) < 1e-4
    p.close()
