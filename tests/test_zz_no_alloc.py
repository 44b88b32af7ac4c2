"""pfe_orthonormalize_noalloc: the allocation-free entry point.

Some callers cannot call cudaMalloc at all: plug-ins inside a host
application that owns every device allocation through its own pool, or
services that size device memory once at start-up.  For them the library
offers one entry point whose scratch memory is a fixed array compiled into
the library.  This test calls it through the C ABI,
twice in a row, and checks it against the D-orthonormalisation that
pfe_init performs (which allocates its own buffers), within the tolerance
the other FP64 tests use.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from oracle import pfe_oracle as O
from tests.gpu_common import gpu_problem, oracle_graph, relerr, small_spec

pytestmark = pytest.mark.gpu


def _noalloc(lib, Y, deg, out, stream_ptr=None):
    f = lib.pfe_orthonormalize_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f(Y.data_ptr(), deg.data_ptr(), Y.shape[0], Y.shape[1], out.data_ptr(), stream_ptr)


def test_noalloc_matches_pfe_init_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_1612_06496_gb300 import load_library
    lib = load_library()
    for call, spec in enumerate([small_spec(H=23, W=29, d=5), small_spec(H=40, W=37, d=9, seed=12)]):
        p, X, Y0 = gpu_problem(spec, "fp64", tol=1e-12)
        p.init(Y0)
        ref = p.get("Y")        # D^{-1/2} polar(D^{1/2} Y0), computed with library-allocated buffers
        deg = p.get("DEG")
        p.close()
        Yd = torch.from_numpy(Y0).cuda()
        degd = torch.from_numpy(deg).cuda()
        out = torch.full_like(Yd, float("nan"))
        torch.cuda.synchronize()
        st = _noalloc(lib, Yd, degd, out, torch.cuda.current_stream().cuda_stream)
        assert st == 0, (call, st)
        got = out.cpu().numpy()
        assert relerr(got, ref) <= 1e-12, call
        # and the defining property: Yhat^T D Yhat = I
        assert np.max(np.abs(got.T @ (deg[:, None] * got) - np.eye(spec.d))) <= 1e-12
        # independent check against the oracle's SVD polar factor
        g = oracle_graph(spec, X)
        assert relerr(got, O.d_orthonormalize(Y0, g.dvec)) <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_1612_06496_gb300 import load_library
    lib = load_library()
    Y = torch.zeros((64, 17), dtype=torch.float64, device="cuda")
    deg = torch.ones(64, dtype=torch.float64, device="cuda")
    out = torch.empty_like(Y)
    assert _noalloc(lib, Y, deg, out) == 1          # d = 17 > 16: PFE_EINVAL
    Yh = np.zeros((64, 3))
    f = lib.pfe_orthonormalize_noalloc
    # host pointers are refused (the entry point copies nothing)
    assert f(Yh.ctypes.data, deg.data_ptr(), 64, 3, out.data_ptr(), None) == 1


def test_noalloc_singular_call_then_a_good_one():
    """A rank-deficient D^{1/2} Y (two equal columns) is PFE_ESINGULAR and
    leaves Yhat as it was; the next call on the same device starts from the
    shared array that call left behind and is exact again."""
    torch = pytest.importorskip("torch")
    from paper_1612_06496_gb300 import load_library
    lib = load_library()
    spec = small_spec(H=19, W=21, d=4, seed=14)
    p, X, Y0 = gpu_problem(spec, "fp64", tol=1e-12)
    p.init(Y0)
    ref = p.get("Y")
    deg = p.get("DEG")
    p.close()
    degd = torch.from_numpy(deg).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    bad = Y0.copy()
    bad[:, 2] = bad[:, 1]
    out = torch.full((spec.n, 4), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert _noalloc(lib, torch.from_numpy(bad).cuda(), degd, out, stream) == 6  # PFE_ESINGULAR
    assert torch.isnan(out).all()
    out2 = torch.full_like(out, float("nan"))
    assert _noalloc(lib, torch.from_numpy(Y0).cuda(), degd, out2, stream) == 0
    assert relerr(out2.cpu().numpy(), ref) <= 1e-12
