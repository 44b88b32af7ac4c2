"""Edge-list graphs on the GPU and the error paths of the C ABI (every
failure is made on the host or through the inputs; nothing faults a GPU)."""

import numpy as np
import pytest

from oracle import pfe_oracle as O
from tests.gpu_common import ensure_built, gpu_problem, relerr, small_spec

pytestmark = pytest.mark.gpu


def _edge_problem(seed=0, n=300, k=6, m=4):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, m))
    # k nearest neighbours (brute force), symmetrised, listed once with a < b
    d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    nn = np.argsort(d2, axis=1)[:, :k]
    pairs = {(min(i, j), max(i, j)) for i in range(n) for j in nn[i]}
    pairs = sorted(pairs)
    a = np.array([p[0] for p in pairs], dtype=np.int32)
    b = np.array([p[1] for p in pairs], dtype=np.int32)
    return X, a, b


def _pfe(X, a, b, sigma, **kw):
    ensure_built()
    from paper_1612_06496_gb300 import PFE
    return PFE(np.ascontiguousarray(X), sigma=sigma, edges=(a, b), **kw)


def test_edge_list_graph_and_solve_match_oracle():
    X, a, b = _edge_problem()
    sigma = 1.2
    rng = np.random.default_rng(1)
    perm = rng.permutation(a.shape[0])          # any order; ids follow the input order
    a, b = a[perm], b[perm]
    flip = rng.uniform(size=a.shape[0]) < 0.5   # either orientation
    ei = np.where(flip, b, a).astype(np.int32)
    ej = np.where(flip, a, b).astype(np.int32)
    p = _pfe(X, ei, ej, sigma, precision="fp64", tol=1e-12)
    g = O.build_graph(X, a.astype(np.int64), b.astype(np.int64), sigma)
    ga, gb, gw = p.edges()
    np.testing.assert_array_equal(ga, a)
    np.testing.assert_array_equal(gb, b)
    np.testing.assert_allclose(gw, g.w, rtol=2e-13)
    np.testing.assert_allclose(p.get("DEG"), g.dvec, rtol=1e-13)
    Y0 = rng.standard_normal((X.shape[0], 4))
    p.init(Y0)
    Y = np.empty((X.shape[0], 4))
    p.solve(3, 4, Y, None)
    st = O.soc_pfe(g, Y0, 3, 4)
    assert relerr(Y, st.Y) <= 1e-9
    # the library clears b when a P-step ends, the oracle when the next outer
    # iteration starts (Alg. 2 step 3): compare b after one more inner step
    assert not np.any(p.get("BS"))
    O.reset_inner(st)
    O.split_bregman_step(g, st, O.DirectSolver(g.A))
    p.inner_step()
    assert relerr(p.get("Y"), st.Y) <= 1e-9
    np.testing.assert_allclose(p.get("BS"), st.bs, atol=1e-9 * max(1.0, np.abs(st.bs).max()))
    p.close()


def test_disconnected_components_are_a_fixed_point():
    """k components and a piecewise-constant D-orthonormal start: M Y = 0, so
    the iteration must return the start exactly (up to FP64 rounding)."""
    rng = np.random.default_rng(13)
    sizes = [40, 55, 33]
    parts, aa, bb, off = [], [], [], 0
    for s in sizes:
        parts.append(rng.standard_normal((s, 3)) + 20 * len(parts))
        for i in range(s - 1):
            aa.append(off + i)
            bb.append(off + i + 1)
        for i in range(0, s - 3, 3):
            aa.append(off + i)
            bb.append(off + i + 3)
        off += s
    X = np.vstack(parts)
    a, b = np.array(aa, dtype=np.int32), np.array(bb, dtype=np.int32)
    labels = np.repeat(np.arange(3), sizes)
    ind = np.stack([(labels == k).astype(float) for k in range(3)], axis=1)
    Y0 = ind[:, :2] - 0.3 * ind[:, 2:3]
    for precision, tol in (("fp64", 1e-12), ("mixed", 2e-6)):
        p = _pfe(X, a, b, 1.5, precision=precision)
        p.init(Y0)
        start = p.get("Y")
        Y = np.empty_like(start)
        p.solve(3, 3, Y, None)
        for k in range(3):
            blk = Y[labels == k]
            assert np.max(np.abs(blk - blk[0])) <= tol * np.max(np.abs(Y)), (precision, k)
        assert relerr(Y, start) <= tol, precision
        p.close()


def test_zero_degree_vertex_is_rejected():
    from paper_1612_06496_gb300 import PFE, PFEError
    ensure_built()
    X = np.zeros((8 * 9, 5))
    X[17] = 1e3            # every weight of vertex 17 underflows to 0
    with pytest.raises(PFEError) as ei:
        PFE(X, sigma=0.1, H=8, W=9, radius=2.0)
    assert ei.value.status == 1
    assert "zero degree" in str(ei.value)  # the build's message outlives its context


@pytest.mark.parametrize("bad", ["self", "dup", "range"])
def test_bad_edge_lists_are_rejected(bad):
    from paper_1612_06496_gb300 import PFEError
    X, a, b = _edge_problem(n=50, k=3)
    a, b = a.copy(), b.copy()
    if bad == "self":
        b[3] = a[3]
    elif bad == "dup":
        a[4], b[4] = b[5], a[5]       # the same pair as edge 5, other orientation
    else:
        b[2] = 50
    with pytest.raises(PFEError) as ei:
        _pfe(X, a, b, 1.0)
    assert ei.value.status == 1
    assert {"self": "self-loop", "dup": "same pair", "range": "outside"}[bad] in str(ei.value)


def test_dimension_and_call_order_errors():
    from paper_1612_06496_gb300 import PFEError, load_library
    spec = small_spec(H=10, W=11, d=3)
    p, X, Y0 = gpu_problem(spec, "mixed")
    with pytest.raises(PFEError) as ei:
        p.inner_step()
    assert ei.value.status == 9                          # PFE_ESTATE before pfe_init
    with pytest.raises(PFEError) as ei:
        p.init(np.zeros((spec.n, 17)))
    assert ei.value.status == 8                          # d = 17 not built in
    lib = load_library()
    assert lib.pfe_init(p.ctx, 3, Y0.ctypes.data, 2) == 1  # ldY0 < d
    assert lib.pfe_init(p.ctx, 40, None, 40) == 8          # d = 40: not built in
    p.close()


def test_singular_start_is_rejected():
    from paper_1612_06496_gb300 import PFEError
    spec = small_spec(H=12, W=12, d=3)
    p, X, Y0 = gpu_problem(spec, "fp64")
    Y0 = Y0.copy()
    Y0[:, 2] = Y0[:, 0]                                   # rank 2
    with pytest.raises(PFEError) as ei:
        p.init(Y0)
    assert ei.value.status == 6
    p.close()


def test_pcg_not_converged_is_reported_and_results_written():
    from paper_1612_06496_gb300 import PFEError
    spec = small_spec(H=14, W=15, d=2)
    p, X, Y0 = gpu_problem(spec, "fp64", tol=1e-14, max_iter=2)
    p.init(Y0)
    Y = np.full((spec.n, 2), np.nan)
    with pytest.raises(PFEError) as ei:
        p.solve(1, 2, Y, None)
    assert ei.value.status == 4
    assert np.all(np.isfinite(Y))
    st = p.solve(1, 1, Y, None, allow_notconv=True)
    assert st["n_unconverged"] == 1 and st["pcg_iters_max"] == 2
    p.close()


def test_nan_right_hand_side_is_reported():
    from paper_1612_06496_gb300 import PFEError
    spec = small_spec(H=14, W=13, d=3)
    for loop in ("graph", "host"):
        p, X, Y0 = gpu_problem(spec, "mixed", loop=loop)
        p.init(Y0)
        rhs = p.get("RHS")
        rhs[7, 1] = np.nan
        p.set("RHS", rhs)
        with pytest.raises(PFEError) as ei:
            p.inner_step(stats=True)
        assert ei.value.status == 5, loop
        p.close()


def test_device_memory_cap():
    """pfe_params.max_device_bytes bounds the memory a context keeps: a build
    or pfe_init that would pass it fails with PFE_ENOMEM and keeps nothing
    of the failed call; the FSAI buffers are all or nothing; a re-init
    returns the previous dimension's buffers."""
    from paper_1612_06496_gb300 import PFE, PFEError
    from synth import make_problem
    ensure_built()
    spec = small_spec(H=14, W=15, d=3)
    X, Y0 = make_problem(spec)
    kw = dict(sigma=spec.sigma, H=14, W=15, radius=spec.radius, precision="mixed")
    p = PFE(X, **kw)
    b_graph = p.info()["device_bytes"]
    p.init(Y0)
    b3 = p.info()["device_bytes"]
    p.init(np.ascontiguousarray(Y0[:, :2]))
    b2 = p.info()["device_bytes"]
    assert b_graph < b2 < b3
    p.close()
    with pytest.raises(PFEError) as ei:
        PFE(X, **kw, max_device_bytes=b_graph // 2)
    assert ei.value.status == 2 and "max_device_bytes" in str(ei.value)
    q = PFE(X, **kw, max_device_bytes=b_graph)
    assert q.info()["device_bytes"] == b_graph
    with pytest.raises(PFEError) as ei:
        q.init(Y0)
    assert ei.value.status == 2 and "max_device_bytes" in str(ei.value)
    assert q.info()["device_bytes"] == b_graph
    with pytest.raises(PFEError) as ei:
        q.inner_step()
    assert ei.value.status == 9  # still not initialised
    q.close()
    # room for the d = 3 state and the first FSAI buffer (G_ii, n floats) only
    r = PFE(X, **kw, max_device_bytes=b3 + 4 * spec.n)
    r.init(Y0)
    assert r.info()["device_bytes"] == b3
    with pytest.raises(PFEError) as ei:
        r.fsai_classical()
    assert ei.value.status == 2
    assert r.info()["device_bytes"] == b3  # the buffer that fitted was released again
    Y = np.empty((spec.n, 3))
    assert r.solve(1, 2, Y, None)["n_unconverged"] == 0  # Jacobi still runs
    r.close()
