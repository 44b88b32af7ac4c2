"""The paper's incomplete-Cholesky preconditioner, IC(0), on the GPU (through
the C ABI) against the FP64 oracle: the factor, PCG iteration counts and
solutions, the graph loop, and the cases it rejects."""
import numpy as np
import pytest

from oracle import ic_oracle as I
from oracle import pfe_oracle as O
from tests.gpu_common import gpu_problem, oracle_graph, relerr, small_spec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("H,W,d,radius", [(23, 29, 3, 2.0), (21, 26, 4, 3.0)])
def test_ic0_factor_matches_oracle(H, W, d, radius):
    spec = small_spec(H=H, W=W, d=d, radius=radius)
    p, X, Y0 = gpu_problem(spec, "mixed")
    g = oracle_graph(spec, X)
    p.init(Y0)
    p.ic0()
    gd, ge = p.fsai_get()
    L = I.ic0(g.A).tocsr()
    # FP64 factor stored as FP32
    np.testing.assert_allclose(gd, L.diagonal(), rtol=2e-7)
    Lba = np.asarray(L[g.b, g.a]).ravel()
    np.testing.assert_allclose(ge, Lba, rtol=2e-6, atol=1e-7 * np.abs(Lba).max())
    p.close()


@pytest.mark.parametrize("H,W,d,radius", [(23, 29, 3, 2.0), (21, 26, 4, 3.0)])
def test_pcg_with_ic0_matches_oracle(H, W, d, radius):
    spec = small_spec(H=H, W=W, d=d, radius=radius)
    p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-6)
    g = oracle_graph(spec, X)
    p.init(Y0)
    rng = np.random.default_rng(31)
    R = rng.standard_normal((g.n, d))
    Yj = np.zeros_like(R)
    it_jacobi = p.solve_system(R, Yj)["pcg_iters"]
    p.ic0()
    Y = np.zeros_like(R)
    st = p.solve_system(R, Y)
    L = I.ic0(g.A).tocsr()
    Yo, info = O.pcg(g.A, R, np.zeros_like(R), 1e-6, 5000, 50, lambda Rm: I.ic0_apply(L, Rm))
    assert st["converged"] and info["converged"]
    assert abs(st["pcg_iters"] - int(info["iters"].max())) <= 2, (st["pcg_iters"], info["iters"])
    assert st["pcg_iters"] < it_jacobi
    assert relerr(Y, Yo) < 1e-4
    assert relerr(Y, O.DirectSolver(g.A)(R)[0]) < 1e-4
    p.close()


def test_ic0_in_the_loop_graph_equals_host():
    """The whole iteration with IC(0): the captured CUDA graph and the
    host-polled loop launch the same kernels and agree bit for bit; the
    result matches the oracle's trajectory with the exact solve."""
    spec = small_spec(H=16, W=20, d=3)
    out = []
    for loop in ("graph", "host"):
        p, X, Y0 = gpu_problem(spec, "mixed", tol=1e-7, loop=loop)
        p.init(Y0)
        p.ic0()
        Y = np.empty_like(Y0)
        st = p.solve(2, 3, Y, None)
        assert st["n_unconverged"] == 0
        out.append(Y)
        p.close()
    np.testing.assert_array_equal(out[0], out[1])
    g = oracle_graph(spec, X)
    ref = O.soc_pfe(g, Y0, 2, 3)
    assert relerr(out[0], ref.Y) < 2e-4


def test_ic0_switches_back_and_rejects_what_it_does_not_cover():
    from paper_1612_06496_gb300 import PFEError
    spec = small_spec(H=14, W=15, d=2)
    p, X, Y0 = gpu_problem(spec, "mixed")
    p.init(Y0)
    R = np.random.default_rng(3).standard_normal((spec.n, 2))
    Y1 = np.zeros_like(R)
    s1 = p.solve_system(R, Y1)
    p.ic0()
    p.fsai_set(None)  # back to Jacobi
    Y2 = np.zeros_like(R)
    s2 = p.solve_system(R, Y2)
    assert s1["pcg_iters"] == s2["pcg_iters"]
    np.testing.assert_array_equal(Y1, Y2)
    p.close()
    q, _, _ = gpu_problem(spec, "fp64")
    with pytest.raises(PFEError) as ei:
        q.ic0()
    assert ei.value.status == 8
    q.close()
