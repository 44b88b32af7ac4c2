"""Batches of independent images in one block-diagonal graph (one launch per
kernel for all of them), against the oracle run on each image alone: every
image keeps its own lambda, PCG scalars, convergence and P-step."""
import numpy as np
import pytest

from oracle import pfe_oracle as O
from synth import ImageSpec, batch_specs, make_problem
from tests.gpu_common import ensure_built, relerr

pytestmark = pytest.mark.gpu

SHAPES = [(13, 17), (20, 11), (9, 24), (16, 16), (7, 31)]


def _specs(d=3, shapes=SHAPES, regions=3):
    return [ImageSpec(f"b{k}", H, W, regions, 0.05, seed=900 + k, radius=2.0, sigma=0.1, d=d)
            for k, (H, W) in enumerate(shapes)]


def _batch(specs, precision, **kw):
    ensure_built()
    from paper_1612_06496_gb300 import PFE
    probs = [make_problem(s) for s in specs]
    X = np.ascontiguousarray(np.vstack([p[0] for p in probs]))
    Y0 = np.ascontiguousarray(np.vstack([p[1] for p in probs]))
    shapes = [s.shape for s in specs]
    pf = PFE(X, sigma=specs[0].sigma, radius=specs[0].radius, shapes=shapes, precision=precision, **kw)
    off = np.concatenate([[0], np.cumsum([s.n for s in specs])])
    return pf, probs, off, Y0


def _oracle(spec, X, Y0, n_outer, n_inner):
    H, W = spec.shape
    g = O.build_grid_graph(X, H, W, spec.radius, spec.sigma)
    return g, O.soc_pfe(g, Y0, n_outer, n_inner, solver="direct")


def test_batch_graph_and_lambdas():
    specs = _specs()
    pf, probs, off, _ = _batch(specs, "fp64")
    goff, lam = pf.segments()
    np.testing.assert_array_equal(goff, off)
    a, b, w = pf.edges()
    seen = 0
    for k, (s, (X, _)) in enumerate(zip(specs, probs)):
        H, W = s.shape
        g = O.build_grid_graph(X, H, W, s.radius, s.sigma)
        sel = (a >= off[k]) & (a < off[k + 1])
        pairs = set(zip((a[sel] - off[k]).tolist(), (b[sel] - off[k]).tolist()))
        assert pairs == set(zip(g.a.tolist(), g.b.tolist()))
        assert np.all(b[sel] < off[k + 1])                 # no edge leaves its image
        np.testing.assert_allclose(w[sel], [g.w[i] for i in _pair_index(g, a[sel] - off[k], b[sel] - off[k])],
                                   rtol=2e-13)
        assert abs(lam[k] - g.lam) <= 1e-13 * g.lam
        seen += int(sel.sum())
    assert seen == a.shape[0]
    pf.close()


def _pair_index(g, a, b):
    idx = {(int(x), int(y)): i for i, (x, y) in enumerate(zip(g.a, g.b))}
    return [idx[(int(x), int(y))] for x, y in zip(a, b)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 2e-4)])
def test_batch_matches_oracle_per_image(precision, tol):
    specs = _specs()
    pf, probs, off, Y0 = _batch(specs, precision, tol=1e-12 if precision == "fp64" else 1e-6)
    pf.init(Y0)
    Y = np.empty_like(Y0)
    Yh = np.empty_like(Y0)
    pf.solve(3, 4, Y, Yh)
    it, rr = pf.segment_stats()
    for k, (s, (X, Y0s)) in enumerate(zip(specs, probs)):
        g, st = _oracle(s, X, Y0s, 3, 4)
        sl = slice(off[k], off[k + 1])
        assert relerr(Y[sl], st.Y) <= tol, (k, relerr(Y[sl], st.Y))
        E = O.embedding(g, st)
        assert relerr(Yh[sl], E) <= tol, k
        # each image is D-orthonormal on its own
        G = Yh[sl].T @ (g.dvec[:, None] * Yh[sl])
        assert np.max(np.abs(G - np.eye(s.d))) <= 1e-10
    assert np.all(rr <= (1e-12 if precision == "fp64" else 1e-6))
    pf.close()


def test_batch_equals_single_image_runs():
    """The same image alone and inside a batch: identical method, only the
    summation order of the reductions differs."""
    from paper_1612_06496_gb300 import PFE
    specs = _specs(d=4)
    pf, probs, off, Y0 = _batch(specs, "fp64", tol=1e-12)
    pf.init(Y0)
    Yb = np.empty_like(Y0)
    pf.solve(2, 3, Yb, None)
    pf.close()
    for k, (s, (X, Y0s)) in enumerate(zip(specs, probs)):
        H, W = s.shape
        p1 = PFE(X, sigma=s.sigma, H=H, W=W, radius=s.radius, precision="fp64", tol=1e-12)
        p1.init(Y0s)
        Y1 = np.empty_like(Y0s)
        p1.solve(2, 3, Y1, None)
        p1.close()
        assert relerr(Yb[off[k]:off[k + 1]], Y1) <= 1e-10, k


def test_batch_images_converge_independently():
    """Images of different size and contrast need different PCG iteration
    counts; each stops on its own and meets the tolerance."""
    specs = _specs(d=3, shapes=[(40, 40), (8, 9), (25, 33)], regions=4)
    pf, probs, off, Y0 = _batch(specs, "mixed", tol=1e-6)
    pf.init(Y0)
    pf.inner_step()
    it, rr = pf.segment_stats()
    assert np.all(rr <= 1e-6)
    assert len(set(it.tolist())) > 1, it
    st = pf.solve(1, 2)
    assert st["n_solves"] == 2 * len(specs)
    assert st["pcg_iters_max"] >= int(it.max()) - 50
    pf.close()


def test_edge_list_batch_and_cross_edges():
    from paper_1612_06496_gb300 import PFE, PFEError
    ensure_built()
    rng = np.random.default_rng(5)
    sizes = [30, 45, 22]
    Xs, aa, bb, off = [], [], [], [0]
    for s in sizes:
        X = rng.standard_normal((s, 3))
        Xs.append(X)
        for i in range(s):
            for j in (i + 1, i + 3):
                if j < s:
                    aa.append(off[-1] + i)
                    bb.append(off[-1] + j)
        off.append(off[-1] + s)
    X = np.vstack(Xs)
    a, b = np.array(aa, dtype=np.int32), np.array(bb, dtype=np.int32)
    Y0 = rng.standard_normal((X.shape[0], 3))
    pf = PFE(X, sigma=1.5, edges=(a, b), seg_off=off, precision="fp64", tol=1e-12)
    pf.init(Y0)
    Y = np.empty_like(Y0)
    pf.solve(2, 3, Y, None)
    for k, s in enumerate(sizes):
        sl = slice(off[k], off[k + 1])
        sel = (a >= off[k]) & (a < off[k + 1])
        g = O.build_graph(Xs[k], (a[sel] - off[k]).astype(np.int64), (b[sel] - off[k]).astype(np.int64), 1.5)
        st = O.soc_pfe(g, Y0[sl], 2, 3)
        assert relerr(Y[sl], st.Y) <= 1e-9, k
    pf.close()
    a2, b2 = a.copy(), b.copy()
    b2[0] = off[1] + 1  # joins segments 0 and 1
    with pytest.raises(PFEError) as ei:
        PFE(X, sigma=1.5, edges=(a2, b2), seg_off=off)
    assert ei.value.status == 1
    with pytest.raises(PFEError) as ei:
        PFE(X, sigma=1.5, edges=(a, b), seg_off=[0, 30, 29, X.shape[0]])  # a segment of < 2 vertices
    assert ei.value.status == 1


@pytest.mark.parametrize("precond", ["learned", "classical"])
def test_batch_fsai_matches_oracle_per_image(precond):
    """The FSAI preconditioner on a batch (one launch per kernel for every
    image, each image's own lambda in the network features, its own PCG
    scalars and convergence): every image against the oracle's exact
    solves, FP32 path, 2e-4; and the factor of each image equals the one the
    image gets alone."""
    from paper_1612_06496_gb300.learned import load_weights
    specs = _specs(d=4)
    pf, probs, off, Y0 = _batch(specs, "mixed", tol=1e-6)
    if precond == "learned":
        pf.fsai_set(load_weights())
    else:
        pf.fsai_classical()
    pf.init(Y0)
    Y = np.empty_like(Y0)
    Yh = np.empty_like(Y0)
    st = pf.solve(2, 3, Y, Yh)
    assert st["n_unconverged"] == 0
    gd_b, ge_b = pf.fsai_get()
    a_b, b_b, _ = pf.edges()
    for k, (s, (X, Y0s)) in enumerate(zip(specs, probs)):
        g, ost = _oracle(s, X, Y0s, 2, 3)
        sl = slice(off[k], off[k + 1])
        assert relerr(Y[sl], ost.Y) <= 2e-4, k
        assert relerr(Yh[sl], O.embedding(g, ost)) <= 2e-4, k
        # the same factor as the image alone
        from paper_1612_06496_gb300 import PFE
        H, W = s.shape
        p1 = PFE(X, sigma=s.sigma, H=H, W=W, radius=s.radius, precision="mixed")
        if precond == "learned":
            p1.fsai_set(load_weights())
        else:
            p1.fsai_classical()
        gd1, ge1 = p1.fsai_get()
        a1, b1, _ = p1.edges()
        p1.close()
        np.testing.assert_allclose(gd_b[sl], gd1, rtol=1e-6)
        # edges matched by their endpoints (the two lists need not share an order)
        at = {(int(x), int(y)): v for x, y, v in zip(a1, b1, ge1)}
        sel = np.nonzero((a_b >= off[k]) & (a_b < off[k + 1]))[0]
        assert len(sel) == len(at)
        ref = np.array([at[(int(a_b[e] - off[k]), int(b_b[e] - off[k]))] for e in sel])
        np.testing.assert_allclose(ge_b[sel], ref, rtol=1e-5, atol=1e-7 * np.abs(ref).max())
    pf.close()


def test_batch_learned_fsai_cuts_iterations_and_images_converge_independently():
    """With the learned factor each image of a batch needs fewer PCG
    iterations than with Jacobi, and images stop on their own."""
    from paper_1612_06496_gb300.learned import load_weights
    specs = _specs(d=4, shapes=[(40, 48), (25, 31), (33, 29)], regions=4)
    its = {}
    for precond in ("jacobi", "learned"):
        pf, probs, off, Y0 = _batch(specs, "mixed", tol=1e-6)
        if precond == "learned":
            pf.fsai_set(load_weights())
        pf.init(Y0)
        pf.solve(1, 2)
        it, rr = pf.segment_stats()
        assert np.all(rr <= 1e-6)
        its[precond] = it
        pf.close()
    assert np.all(its["learned"] < its["jacobi"]), its


def test_batch_rejects_ic0_and_training():
    from paper_1612_06496_gb300 import PFEError
    from paper_1612_06496_gb300.learned import init_params
    pf, probs, off, Y0 = _batch(_specs(), "mixed")
    with pytest.raises(PFEError) as ei:
        pf.ic0()
    assert ei.value.status == 8
    with pytest.raises(PFEError) as ei:
        pf.fsai_loss_grad(init_params(0))
    assert ei.value.status == 8
    pf.close()


@pytest.mark.parametrize("precond", ["jacobi", "learned"])
def test_c3_batch_full_size(precond):
    """The 64-image batch (96..481 x 96..321, 3-12 regions, radius 2, d = 5),
    with Jacobi and with the learned factor (the benchmark's batch arms):
    one outer iteration of two inner steps; every image converged and
    D-orthonormal, the two smallest images against the oracle."""
    from paper_1612_06496_gb300.learned import load_weights
    specs = batch_specs()
    pf, probs, off, Y0 = _batch(specs, "mixed", tol=1e-6)
    assert pf.info()["nseg"] == 64
    if precond == "learned":
        pf.fsai_set(load_weights())
    pf.init(Y0)
    Y = np.empty_like(Y0)
    Yh = np.empty_like(Y0)
    st = pf.solve(1, 2, Y, Yh)
    assert st["n_unconverged"] == 0 and st["n_solves"] == 2 * 64
    deg = pf.get("DEG")
    for k in range(64):
        sl = slice(off[k], off[k + 1])
        G = Yh[sl].T @ (deg[sl, None] * Yh[sl])
        assert np.max(np.abs(G - np.eye(5))) <= 1e-9, k
    for k in np.argsort([s.n for s in specs])[:2]:
        s, (X, Y0s) = specs[k], probs[k]
        g, ost = _oracle(s, X, Y0s, 1, 2)
        assert relerr(Y[off[k]:off[k + 1]], ost.Y) <= 2e-4, k
    pf.close()
