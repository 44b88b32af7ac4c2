"""Entry points used one at a time, as a caller driving the loop itself
would: pfe_pstep (Alg. 1 steps 6-7 on their own) after inner steps, and
pfe_set_stream moving later work to another stream."""
import numpy as np
import pytest

from oracle import pfe_oracle as O
from synth import make_problem
from tests.gpu_common import gpu_problem, oracle_graph, relerr, small_spec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pstep_closes_an_outer_iteration(precision):
    """Three pfe_inner_step calls, then pfe_pstep, against the oracle's own
    trajectory from the same start: P = polar(D^{1/2} Y + B) and
    B = B + D^{1/2} Y - P (P and B are FP64 in both paths), and b restarted
    at zero for the next outer iteration."""
    spec = small_spec(H=20, W=26, d=3)
    p, X, Y0 = gpu_problem(spec, precision, tol=1e-12 if precision == "fp64" else 1e-6)
    g = oracle_graph(spec, X)
    p.init(Y0)
    st = O.init_state(g, Y0)
    solve = O.DirectSolver(g.A)
    for _ in range(3):
        p.inner_step()
        O.split_bregman_step(g, st, solve)
    p.pstep()
    O.p_and_b_step(g, st)
    tol = 1e-9 if precision == "fp64" else 2e-4
    P, B = p.get("P"), p.get("B")
    assert relerr(P, st.P) <= tol
    # B = X - P is a difference, so its error is taken at the scale of P (|P|_F = sqrt(d))
    assert np.linalg.norm(B - st.B) <= 2 * tol * np.linalg.norm(st.P)
    assert np.max(np.abs(P.T @ P - np.eye(spec.d))) <= 1e-10
    assert not np.any(p.get("BS"))
    p.close()


def test_set_stream_moves_later_work():
    """A context built on the current stream, then moved to a new one before
    its solve, gives bit for bit the result of a context that never moved;
    moving it again after queued work keeps that work first."""
    torch = pytest.importorskip("torch")
    spec = small_spec(H=16, W=18, d=3)
    X, Y0 = make_problem(spec)
    out = []
    for moves in (0, 1, 2):
        p, _, _ = gpu_problem(spec, "fp64", tol=1e-12)
        streams = [torch.cuda.Stream() for _ in range(moves)]
        p.init(Y0)
        if moves >= 1:
            p.set_stream(streams[0])
        if moves == 2:
            p.inner_step()                 # queued on the first new stream
            p.set_stream(streams[1])
            p.pstep()
            p.solve(1, 3)
            Y = p.get("Y")
        else:
            p.inner_step()
            p.pstep()
            p.solve(1, 3)
            Y = p.get("Y")
        out.append(Y)
        p.close()
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(out[0], out[2])
    # the same schedule in the oracle: one inner step and a P-step, then an
    # outer iteration of three inner steps (b restarts at each outer iteration)
    g = oracle_graph(spec, X)
    st = O.init_state(g, Y0)
    solve = O.DirectSolver(g.A)
    O.split_bregman_step(g, st, solve)
    O.p_and_b_step(g, st)
    O.reset_inner(st)
    for _ in range(3):
        O.split_bregman_step(g, st, solve)
    O.p_and_b_step(g, st)
    assert relerr(out[0], st.Y) <= 1e-9
