"""Objective |M Y|_1 and constraint distance |Y^T D Y - I|_F on the GPU
against the oracle, for one image and for a batch."""
import numpy as np
import pytest

from oracle import pfe_oracle as O
from synth import CONFIGS, ImageSpec, make_problem
from tests.gpu_common import ensure_built, gpu_problem, oracle_graph

pytestmark = pytest.mark.gpu


def _fro(Y, dvec):
    return float(np.linalg.norm(Y.T @ (dvec[:, None] * Y) - np.eye(Y.shape[1])))


def test_objective_and_constraint_c1():
    spec = CONFIGS["C1"]
    p, X, Y0 = gpu_problem(spec, "fp64", tol=1e-12)
    g = oracle_graph(spec, X)
    p.init(Y0)
    Y = np.empty_like(Y0)
    p.solve(2, 3, Y, None)
    st = O.soc_pfe(g, Y0, 2, 3)
    E = O.embedding(g, st)
    l1, oe = p.objective("yhat")
    assert abs(l1 - O.objective(g, E)) <= 1e-9 * O.objective(g, E)
    assert oe <= 1e-10
    l1y, oey = p.objective("y")
    assert abs(l1y - O.objective(g, st.Y)) <= 1e-9 * O.objective(g, st.Y)
    assert abs(oey - _fro(st.Y, g.dvec)) <= 1e-8 * max(1.0, _fro(st.Y, g.dvec))
    p.close()


def test_objective_batch_sums_and_max():
    from paper_1612_06496_gb300 import PFE
    ensure_built()
    specs = [ImageSpec(f"o{k}", H, W, 3, 0.05, seed=700 + k, radius=2.0, sigma=0.1, d=3)
             for k, (H, W) in enumerate([(12, 15), (17, 9), (10, 10)])]
    probs = [make_problem(s) for s in specs]
    X = np.ascontiguousarray(np.vstack([q[0] for q in probs]))
    Y0 = np.ascontiguousarray(np.vstack([q[1] for q in probs]))
    pf = PFE(X, sigma=0.1, radius=2.0, shapes=[s.shape for s in specs], precision="fp64", tol=1e-12)
    pf.init(Y0)
    Y = np.empty_like(Y0)
    pf.solve(1, 2, Y, None)
    off = np.concatenate([[0], np.cumsum([s.n for s in specs])])
    tot, worst = 0.0, 0.0
    for k, (s, (Xs, Y0s)) in enumerate(zip(specs, probs)):
        g = O.build_grid_graph(Xs, s.H, s.W, s.radius, s.sigma)
        st = O.soc_pfe(g, Y0s, 1, 2)
        tot += O.objective(g, st.Y)
        worst = max(worst, _fro(st.Y, g.dvec))
    l1, oe = pf.objective("y")
    assert abs(l1 - tot) <= 1e-9 * tot
    assert abs(oe - worst) <= 1e-8 * max(worst, 1.0)
    pf.close()
