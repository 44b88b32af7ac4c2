"""Residual replacement in the PCG of Sec. III and the residual against the
FP64 system matrix of Eq. 13.

The FP32 recurrence r -= alpha q drifts from b - A y by about eps |r_0|; a
warm-started solve (|r_0| ~ 160 |b| on the benchmark image's windows) would
otherwise stop with b - A y about 15x above the tolerance.  The library
freezes a column only on a replaced (true) residual computed with A's FP64
values, so the stated tolerance holds against the problem's matrix."""
import numpy as np
import pytest

from oracle import pfe_oracle as O
from synth import CONFIGS, crop_specs, make_problem
from tests.gpu_common import ensure_built, gpu_problem, oracle_graph, relerr, small_spec

pytestmark = pytest.mark.gpu


def _oracle_relres(A, B, X):
    r = np.linalg.norm(B - A @ X, axis=0)
    b = np.linalg.norm(B, axis=0)
    return np.where(b > 0, r / np.where(b > 0, b, 1.0), r)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_residual_matches_oracle(precision):
    """pfe_residual: FP64 A whatever the context's precision, host and
    device arrays, a zero column (absolute norm)."""
    import torch
    spec = small_spec(H=19, W=23, d=5)
    p, X, Y0 = gpu_problem(spec, precision)
    g = oracle_graph(spec, X)
    p.init(Y0)
    rng = np.random.default_rng(5)
    B = rng.standard_normal((g.n, 5))
    B[:, 3] = 0.0
    Xs = rng.standard_normal((g.n, 5))
    want = _oracle_relres(g.A, B, Xs)
    got = p.residual(B, Xs)
    assert got.shape == (1, 5)
    np.testing.assert_allclose(got[0], want, rtol=1e-12)
    got_d = p.residual(torch.from_numpy(B).cuda(), torch.from_numpy(Xs).cuda())
    np.testing.assert_allclose(got_d[0], want, rtol=1e-12)
    p.close()


def test_residual_per_problem_of_a_batch():
    from paper_1612_06496_gb300 import PFE
    ensure_built()
    specs = [small_spec(H=13, W=17, d=3, seed=21), small_spec(H=20, W=11, d=3, seed=22),
             small_spec(H=9, W=30, d=3, seed=23)]
    probs = [make_problem(s) for s in specs]
    Xf = np.ascontiguousarray(np.vstack([q[0] for q in probs]))
    Y0 = np.ascontiguousarray(np.vstack([q[1] for q in probs]))
    p = PFE(Xf, sigma=0.1, radius=2.0, shapes=[s.shape for s in specs], precision="mixed")
    p.init(Y0)
    rng = np.random.default_rng(6)
    B = rng.standard_normal(Y0.shape)
    Xs = rng.standard_normal(Y0.shape)
    got = p.residual(B, Xs)
    off, lam = p.segments()
    for s, (spec, (Xi, _)) in enumerate(zip(specs, probs)):
        g = O.build_grid_graph(Xi, spec.H, spec.W, spec.radius, spec.sigma, lam=lam[s])
        sl = slice(off[s], off[s + 1])
        np.testing.assert_allclose(got[s], _oracle_relres(g.A, B[sl], Xs[sl]), rtol=1e-12)
    p.close()


def _first_system(spec, precond, **kw):
    """The first inner step's system of Eq. 13 after pfe_init (b = RHS, warm
    start y0 = the D-orthonormalised start)."""
    from paper_1612_06496_gb300.learned import load_weights
    p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-6, **kw)
    if precond == "learned":
        p.fsai_set(load_weights())
    elif precond == "classical":
        p.fsai_classical()
    p.init(Y0)
    return p, X, p.get("RHS"), p.get("Y")


@pytest.mark.parametrize("precond", ["jacobi", "learned", "classical"])
@pytest.mark.parametrize("crop_idx", [0, 3])
def test_warm_started_solve_meets_tol_against_fp64_A(precond, crop_idx):
    """A warm-started FP32 solve at d = 10 (r_0 ~ 160 b): converged, and
    |b - A y| / |b| <= tol with A in FP64 (pfe_residual), as the solve's own
    statistic says.  On this system the learned factor stalled at 2.8e-5
    before replacements were tied to the residual's fall."""
    spec = crop_specs(CONFIGS["C5"])[crop_idx]
    p, X, b, y0 = _first_system(spec, precond)
    g = oracle_graph(spec, X)
    assert _oracle_relres(g.A, b, y0).min() > 100.0  # the start is far from the solution
    Y = y0.copy()
    st = p.solve_system(b, Y)
    assert st["converged"] and st["relres_max"] <= 1e-6
    rel = p.residual(b, Y)[0]
    assert rel.max() <= 1e-6 * (1 + 1e-3), rel
    np.testing.assert_allclose(rel, _oracle_relres(g.A, b, Y), rtol=1e-9)
    p.close()


def test_without_replacement_the_recurrence_stops_short():
    """refresh = 0 turns replacement off: the recurrence residual reaches the
    tolerance while b - A y stays an order of magnitude above it (the drift
    the replacements remove)."""
    spec = crop_specs(CONFIGS["C5"])[3]
    p, X, b, y0 = _first_system(spec, "learned", refresh=0)
    Y = y0.copy()
    st = p.solve_system(b, Y)
    assert st["converged"] and st["relres_max"] <= 1e-6
    assert p.residual(b, Y).max() > 5e-6
    p.close()


def test_paper_scale_image_true_residual():
    """The 481x321 image (radius 3, d = 8) with the learned factor and the
    autotuned SpMM: one outer iteration, then the next system solved from
    its warm start; every column's |b - A y| / |b| <= 1e-6 with A in FP64."""
    from paper_1612_06496_gb300.learned import load_weights
    spec = CONFIGS["C2"]
    p, X, Y0 = gpu_problem(spec, "mixed", tol=spec.tol)
    p.fsai_set(load_weights())
    p.init(Y0)
    p.autotune(5)
    st = p.solve(1, 2)
    assert st["n_unconverged"] == 0 and st["relres_max"] <= 1e-6
    b, Y = p.get("RHS"), p.get("Y")
    s2 = p.solve_system(b, Y)
    assert s2["converged"]
    assert p.residual(b, Y).max() <= 1e-6 * (1 + 1e-3)
    p.close()


@pytest.mark.parametrize("precond", ["jacobi", "learned"])
def test_graph_loop_with_conditional_replacements_equals_host_loop(precond):
    """The captured loop launches the replacement kernels only on
    replacement iterations (conditional IF nodes); the host loop launches
    them every iteration and they return at once.  Same iterations, bit for
    bit, and fewer launches in the graph."""
    from paper_1612_06496_gb300.learned import load_weights
    spec = crop_specs(CONFIGS["C5"])[1]
    out = []
    for loop in ("graph", "host"):
        p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-6, loop=loop)
        if precond == "learned":
            p.fsai_set(load_weights())
        p.init(Y0)
        Y = np.empty_like(Y0)
        s = p.solve(2, 3, Y, None)
        out.append((Y, s))
        p.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1]["pcg_iters_total"] == out[1][1]["pcg_iters_total"]
    assert out[0][1]["kernel_launches"] < out[1][1]["kernel_launches"]
    assert relerr(out[0][0], out[1][0]) == 0.0
