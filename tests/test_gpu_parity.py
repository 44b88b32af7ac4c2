"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: relative Frobenius error of Y <= 1e-9 for the FP64
path (PCG run to relative residual 1e-12, so the iterative solve is
indistinguishable from the oracle's exact solve) and <= 2e-4 for the mixed
path."""
import numpy as np
import pytest

from oracle import pfe_oracle as O
from synth import CONFIGS, make_problem
from tests.gpu_common import gpu_problem, oracle_graph, oracle_run, relerr, small_spec

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
MIXED_TOL = 2e-4


# ---------------------------------------------------------------- graph build


@pytest.mark.parametrize("spec", [small_spec(), small_spec(H=32, W=32, radius=3.0, d=3), CONFIGS["C1"]])
def test_graph_matches_oracle(spec):
    p, X, _ = gpu_problem(spec, "fp64")
    g = oracle_graph(spec, X)
    a, b, w = p.edges()
    np.testing.assert_array_equal(a, g.a)          # index work: bit-exact
    np.testing.assert_array_equal(b, g.b)
    # exp(-u) carries the rounding of u = |x_i - x_j|^2 / (2 sigma^2) with
    # condition number u; u < 745 for any representable weight, so the two
    # summation orders of u may differ by up to ~745 * 2.2e-16 relative
    np.testing.assert_allclose(w, g.w, rtol=2e-13, atol=1e-300)
    np.testing.assert_allclose(p.get("DEG"), g.dvec, rtol=1e-13)
    info = p.info()
    assert info["n_edges"] == g.n_edges
    assert info["lambda_"] == pytest.approx(g.lam, rel=1e-13)
    np.testing.assert_allclose(p.get("DIAG"), g.A.diagonal(), rtol=1e-13)
    p.close()


def test_c2_graph_counts():
    spec = CONFIGS["C2"]
    X, _ = make_problem(spec)
    from paper_1612_06496_gb300 import PFE
    p = PFE(X, sigma=spec.sigma, H=spec.H, W=spec.W, radius=spec.radius, precision="mixed")
    info = p.info()
    assert info["n_edges"] == 2147196 and info["nnz_A"] == 4448793
    g = oracle_graph(spec, X)
    np.testing.assert_allclose(p.get("DEG"), g.dvec, rtol=1e-12)
    a, b, w = p.edges()
    np.testing.assert_array_equal(a, g.a)
    np.testing.assert_array_equal(b, g.b)
    np.testing.assert_allclose(w, g.w, rtol=2e-13, atol=1e-300)
    p.close()


# ---------------------------------------------------------------- operators


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 3e-6)])
@pytest.mark.parametrize("d", [1, 3, 5, 8, 10])
def test_apply_A(precision, tol, d):
    spec = small_spec(H=19, W=23, d=d)
    p, X, Y0 = gpu_problem(spec, precision)
    g = oracle_graph(spec, X)
    p.init(Y0)
    rng = np.random.default_rng(d)
    Z = rng.standard_normal((g.n, d))
    out = p.apply_A(Z)
    assert relerr(out, g.A @ Z) < tol
    p.close()


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-9), ("mixed", 1e-6, 1e-4)])
def test_solve_system_matches_direct(precision, tol, bound):
    spec = small_spec(H=24, W=29, d=4)
    p, X, Y0 = gpu_problem(spec, precision, tol=tol)
    g = oracle_graph(spec, X)
    p.init(Y0)
    rng = np.random.default_rng(3)
    R = rng.standard_normal((g.n, 4))
    Y = np.zeros_like(R)
    st = p.solve_system(R, Y)
    assert st["converged"] and st["pcg_iters"] > 0
    Yd = O.DirectSolver(g.A)(R)[0]
    assert relerr(Y, Yd) < bound
    # the true residual reaches the tolerance
    res = np.linalg.norm(R - g.A @ Y, axis=0) / np.linalg.norm(R, axis=0)
    assert res.max() < 3 * tol
    p.close()


# ---------------------------------------------------------------- init / P-step


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_init_d_orthonormalises(precision):
    spec = small_spec(H=21, W=22, d=6)
    p, X, Y0 = gpu_problem(spec, precision)
    g = oracle_graph(spec, X)
    p.init(Y0)
    Yg = p.get("Y")
    Yo = O.d_orthonormalize(Y0, g.dvec)
    assert relerr(Yg, Yo) < (1e-12 if precision == "fp64" else 1e-7)
    P = p.get("P")
    np.testing.assert_allclose(P.T @ P, np.eye(6), atol=1e-12)
    assert np.all(p.get("B") == 0)
    p.close()


# ---------------------------------------------------------------- one inner step


def test_single_inner_step_state_fp64():
    spec = small_spec(H=20, W=26, d=3)
    p, X, Y0 = gpu_problem(spec, "fp64", tol=1e-12)
    g = oracle_graph(spec, X)
    p.init(Y0)
    st = O.init_state(g, Y0)
    solve = O.DirectSolver(g.A)
    for step in range(3):
        p.inner_step()
        O.split_bregman_step(g, st, solve)
        assert relerr(p.get("Y"), st.Y) < 1e-9, step
        assert relerr(p.get("BS"), st.bs) < 1e-8, step
        rhs_next = g.lam * (g.M.T @ (st.ds - st.bs)) + g.r * np.sqrt(g.dvec)[:, None] * (st.P - st.B)
        assert relerr(p.get("RHS"), rhs_next) < 1e-9, step
    p.close()


def test_single_inner_step_state_mixed():
    """The FP32 path's edge pass against the oracle, element by element, with
    bounds that follow from the method.  The Bregman update of Eq. 10 is
    b' = b + E - Shrink(E + b, 1/lam) = clamp(E + b, -1/lam, 1/lam), a
    1-Lipschitz map of t = E + b (no jump where the shrink switches on), and
    E_e = w_e (y_a - y_b).  So an error dY in the solve (bounded by the PCG
    tolerance, 2e-4 relative) moves b'_e by at most
    T_e = w_e (|dy_a| + |dy_b|) + (the bound on b_e) + FP32 rounding, and the
    next right-hand side lam M^T (Z - b') + r D^{1/2} (P - B), Z - b' = t -
    2 clamp(t), by at most lam sum over the row's edges of 3 w_e T_e plus
    rounding.  Differences of nearby y are small in smooth regions, so these
    errors can be large relative to b and the right-hand side (the norm
    errors are also printed) while every element stays inside its bound."""
    spec = small_spec(H=20, W=26, d=3)
    p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-6)
    g = oracle_graph(spec, X)
    p.init(Y0)
    st = O.init_state(g, Y0)
    solve = O.DirectSolver(g.A)
    u32 = 2.0 ** -24
    gam = 1.0 / g.lam
    absM = abs(g.M)
    sq = np.sqrt(g.dvec)[:, None]
    Tb = np.zeros_like(st.bs)  # bound on |db| entering the step
    for step in range(3):
        b_old = st.bs.copy()
        p.inner_step()
        O.split_bregman_step(g, st, solve)
        Yg = p.get("Y")
        assert relerr(Yg, st.Y) < 2e-4, step
        dy = np.abs(Yg - st.Y)
        w = g.w[:, None]
        E = g.M @ st.Y
        # FP32 rounding of y (hi part), w, the difference, the product and t = E + b
        rnd = 8 * u32 * (w * (np.abs(st.Y[g.a]) + np.abs(st.Y[g.b])) + np.abs(b_old) + np.abs(E) + gam)
        Tt = w * (dy[g.a] + dy[g.b]) + Tb + rnd
        bg = p.get("BS")
        err_b = np.abs(bg - st.bs)
        assert np.all(err_b <= Tt), (step, float(np.max(err_b / Tt)))
        Tb = Tt
        q = st.ds - st.bs  # Z - b'
        C = g.r * sq * (st.P - st.B)
        rhs_next = g.lam * (g.M.T @ q) + C
        # 12 or fewer FP32 terms a row, each rounded, and C's FP32 rounding
        rnd_r = 32 * u32 * (g.lam * (absM.T @ np.abs(q)) + np.abs(C))
        Tr = g.lam * (absM.T @ (3 * Tt)) + rnd_r
        err_r = np.abs(p.get("RHS") - rhs_next)
        assert np.all(err_r <= Tr), (step, float(np.max(err_r / Tr)))
        print(f"step {step}: relerr Y {relerr(Yg, st.Y):.2e} b {relerr(bg, st.bs):.2e} "
              f"rhs {relerr(p.get('RHS'), rhs_next):.2e}; worst element / bound: b "
              f"{np.max(err_b / Tt):.2f}, rhs {np.max(err_r / Tr):.2f}")
    p.close()


# ---------------------------------------------------------------- whole solve


def test_c1_fp64_full_solve_parity():
    spec = CONFIGS["C1"]
    g, st, Yh = oracle_run("C1", spec.n_outer, spec.n_inner)
    p, X, Y0 = gpu_problem(spec, "fp64", tol=1e-12)
    p.init(Y0)
    Y = np.empty((spec.n, spec.d))
    Yhat = np.empty((spec.n, spec.d))
    stats = p.solve(spec.n_outer, spec.n_inner, Y, Yhat)
    assert stats["n_unconverged"] == 0 and stats["n_solves"] == spec.n_outer * spec.n_inner
    assert relerr(Y, st.Y) <= FP64_TOL
    assert relerr(Yhat, Yh) <= FP64_TOL
    assert np.max(np.abs(Yhat.T @ (g.dvec[:, None] * Yhat) - np.eye(spec.d))) <= 1e-10
    p.close()


def test_c1_config_tolerance_parity():
    """At C1's own PCG tolerance (1e-8) the FP64 path still meets 1e-9."""
    spec = CONFIGS["C1"]
    g, st, Yh = oracle_run("C1", spec.n_outer, spec.n_inner)
    p, X, Y0 = gpu_problem(spec, "fp64", tol=spec.tol)
    p.init(Y0)
    Y = np.empty((spec.n, spec.d))
    p.solve(spec.n_outer, spec.n_inner, Y, None)
    assert relerr(Y, st.Y) <= FP64_TOL
    p.close()


def test_c1_mixed_full_solve_parity():
    spec = CONFIGS["C1"]
    g, st, Yh = oracle_run("C1", spec.n_outer, spec.n_inner)
    p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-6)
    p.init(Y0)
    Y = np.empty((spec.n, spec.d))
    Yhat = np.empty((spec.n, spec.d))
    p.solve(spec.n_outer, spec.n_inner, Y, Yhat)
    assert relerr(Y, st.Y) <= MIXED_TOL
    assert relerr(Yhat, Yh) <= MIXED_TOL
    assert np.max(np.abs(Yhat.T @ (g.dvec[:, None] * Yhat) - np.eye(spec.d))) <= 1e-10
    p.close()


@pytest.mark.parametrize("crop_idx", [0, 1, 2, 3])
def test_c5_crops_parity(crop_idx):
    """The large image's generator, checked on seeded 64x64 windows (d = 10)."""
    from synth import crop_specs
    spec = crop_specs(CONFIGS["C5"])[crop_idx]
    X, Y0 = make_problem(spec)
    g = oracle_graph(spec, X)
    ost = O.soc_pfe(g, Y0, 3, 5, solver="direct")
    for precision, tol, bound in (("fp64", 1e-12, FP64_TOL), ("mixed", 1e-6, MIXED_TOL)):
        p, _, _ = gpu_problem(spec, precision, tol=tol)
        p.init(Y0)
        Y = np.empty((spec.n, spec.d))
        Yhat = np.empty((spec.n, spec.d))
        p.solve(3, 5, Y, Yhat)
        assert relerr(Y, ost.Y) <= bound, precision
        assert relerr(Yhat, O.embedding(g, ost)) <= bound, precision
        p.close()


@pytest.mark.parametrize("d", [1, 2, 5, 7])
def test_ragged_sizes_and_odd_d(d):
    """n not a multiple of 32, odd d, radius 3 boundary rows."""
    spec = small_spec(H=11, W=13, d=d, radius=3.0)
    X, Y0 = make_problem(spec)
    g = oracle_graph(spec, X)
    ost = O.soc_pfe(g, Y0, 2, 3, solver="direct")
    p, _, _ = gpu_problem(spec, "fp64", tol=1e-12)
    p.init(Y0)
    Y = np.empty((spec.n, d))
    p.solve(2, 3, Y, None)
    assert relerr(Y, ost.Y) <= FP64_TOL
    p.close()


def test_loop_modes_identical():
    """The CUDA-graph WHILE loop and the host poll loop run the same kernels."""
    spec = small_spec(H=30, W=31, d=4)
    out = []
    for loop in ("graph", "host"):
        p, X, Y0 = gpu_problem(spec, "mixed", loop=loop, check_every=3)
        p.init(Y0)
        Y = np.empty((spec.n, 4))
        s = p.solve(2, 4, Y, None)
        out.append((Y, s["pcg_iters_total"]))
        p.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_checkpoint_resume_bitwise():
    spec = small_spec(H=25, W=27, d=3)
    p, X, Y0 = gpu_problem(spec, "mixed")
    p.init(Y0)
    for _ in range(3):
        p.inner_step()
    state = {k: p.get(k) for k in ("Y", "P", "B", "BS", "RHS")}
    for _ in range(2):
        p.inner_step()
    ref = p.get("Y")
    q, _, _ = gpu_problem(spec, "mixed")
    q.init(Y0)
    for k, v in state.items():
        q.set(k, v)
    for _ in range(2):
        q.inner_step()
    # the FP64 round trip of the FP32 hi/lo pair is exact, so the runs agree bitwise
    np.testing.assert_array_equal(q.get("Y"), ref)
    p.close()
    q.close()


def test_device_pointers_and_torch_stream():
    torch = pytest.importorskip("torch")
    spec = small_spec(H=16, W=18, d=3)
    X, Y0 = make_problem(spec)
    from paper_1612_06496_gb300 import PFE
    s = torch.cuda.Stream()
    Xd = torch.from_numpy(X).cuda()
    Y0d = torch.from_numpy(Y0).cuda()
    with torch.cuda.stream(s):
        p = PFE(Xd, sigma=spec.sigma, H=16, W=18, radius=spec.radius, precision="fp64", tol=1e-12, stream=s)
        p.init(Y0d)
        Yd = torch.empty((spec.n, 3), dtype=torch.float64, device="cuda")
        p.solve(2, 3, Yd, None)
    s.synchronize()
    g = oracle_graph(spec, X)
    ost = O.soc_pfe(g, Y0, 2, 3, solver="direct")
    assert relerr(Yd.cpu().numpy(), ost.Y) <= FP64_TOL
    p.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 2e-4)])
def test_two_stage_schedule(precision, tol):
    """Sec. IV: Stage I (SOC) then Stage II (split Bregman with P, B held)."""
    spec = CONFIGS["C1"]
    p, X, Y0 = gpu_problem(spec, precision, tol=1e-12 if precision == "fp64" else 1e-6)
    g = oracle_graph(spec, X)
    p.init(Y0)
    Y = np.empty_like(Y0)
    Yh = np.empty_like(Y0)
    st = p.solve_two_stage(3, 5, 12, Y, Yh)
    assert st["n_solves"] == 3 * 5 + 12
    ost = O.two_stage(g, Y0, 3, 5, 12)
    assert relerr(Y, ost.Y) <= tol
    assert relerr(Yh, O.embedding(g, ost)) <= tol
    p.close()
