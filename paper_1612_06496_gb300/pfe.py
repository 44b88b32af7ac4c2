"""ctypes binding of libpfe (include/pfe.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
they must be C-contiguous float64 (int32 for edge lists).  Importing this
module raises if libpfe.so has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpfe.so")

PFE_OK, PFE_EINVAL, PFE_ENOMEM, PFE_ECUDA, PFE_ENOTCONV, PFE_ENUMERIC, PFE_ESINGULAR, PFE_ETIMEOUT, \
    PFE_EUNSUPPORTED, PFE_ESTATE = range(10)
PFE_GRAPH_GRID, PFE_GRAPH_EDGES = 0, 1
PFE_FP64, PFE_MIXED = 0, 1
PFE_PRECOND_JACOBI = 0
PFE_LOOP_GRAPH, PFE_LOOP_HOST = 0, 1
ARR = {"Y": 0, "P": 1, "B": 2, "BS": 3, "RHS": 4, "DEG": 5, "DIAG": 6}

EXPORTS = ["pfe_default_params", "pfe_build_graph", "pfe_init", "pfe_inner_step", "pfe_pstep", "pfe_solve",
           "pfe_destroy", "pfe_last_error", "pfe_status_string", "pfe_get_info", "pfe_set_stream",
           "pfe_get_array", "pfe_set_array", "pfe_get_edges", "pfe_apply_A", "pfe_solve_system",
           "pfe_time_kernel", "pfe_fsai_param_count", "pfe_fsai_set", "pfe_fsai_loss_grad", "pfe_fsai_loss_grad_rhs", "pfe_fsai_get",
           "pfe_adam_update", "pfe_orthonormalize_noalloc", "pfe_fsai_classical", "pfe_ic0", "pfe_get_segments",
           "pfe_get_segment_stats", "pfe_laplacian_eigenmap", "pfe_objective", "pfe_autotune",
           "pfe_set_variant", "pfe_solve_two_stage", "pfe_kmeans", "pfe_residual", "pfe_get_variant",
           "pfe_get_shape", "pfe_set_shape"]
SPMM_NVARIANTS = 8  # PFE_SPMM_GENERAL, _ROW1, _ROW2, _ROW2_4, _TMA, _STENCIL, _GRID1, _GRID2
TUNE = {"spmm": 0, "fsai": 1, "edge": 2, "mlp": 3}
KERNEL = {"spmm": 0, "update": 1, "edge": 2, "pupdate": 3, "fsai_tr": 4, "fsai_zp": 5, "fsai_zp_hold": 6,
          "pupdate_hold": 7, "replace": 8, "xflush": 9, "fsai_t": 10, "mlp": 11}


class GraphDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int32), ("kind", C.c_int32), ("features", C.c_void_p),
                ("H", C.c_int32), ("W", C.c_int32), ("radius", C.c_double),
                ("ei", C.c_void_p), ("ej", C.c_void_p), ("n_edges", C.c_int64), ("sigma", C.c_double),
                ("nseg", C.c_int32), ("seg_hw", C.c_void_p), ("seg_off", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("r", C.c_double), ("precision", C.c_int32), ("precond", C.c_int32),
                ("tol", C.c_double), ("max_iter", C.c_int32), ("refresh", C.c_int32),
                ("reset_inner_each_outer", C.c_int32), ("loop_mode", C.c_int32), ("check_every", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("max_device_bytes", C.c_int64)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_edges", C.c_int64), ("nnz_A", C.c_int64), ("sell_slots", C.c_int64),
                ("d", C.c_int32), ("precision", C.c_int32), ("lambda_", C.c_double), ("r", C.c_double),
                ("vol", C.c_double), ("device_bytes", C.c_int64), ("nseg", C.c_int32), ("le_iters", C.c_int32),
                ("le_residual", C.c_double)]


class StepStats(C.Structure):
    _fields_ = [("pcg_iters", C.c_int32), ("converged", C.c_int32), ("relres_max", C.c_double)]


class SolveStats(C.Structure):
    _fields_ = [("pcg_iters_total", C.c_int64), ("pcg_iters_max", C.c_int32), ("n_solves", C.c_int32),
                ("n_unconverged", C.c_int32), ("relres_max", C.c_double), ("kernel_launches", C.c_int64),
                ("pcg_rounds", C.c_int64), ("replacements", C.c_int64)]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libpfe.so (raises OSError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libpfe.so not found at {path}; run `python -m paper_1612_06496_gb300.build`")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.pfe_default_params.argtypes = [C.POINTER(Params)]
    lib.pfe_default_params.restype = None
    lib.pfe_build_graph.argtypes = [C.POINTER(vp), C.POINTER(GraphDesc), C.POINTER(Params), vp]
    lib.pfe_init.argtypes = [vp, i32, vp, i64]
    lib.pfe_inner_step.argtypes = [vp, C.POINTER(StepStats)]
    lib.pfe_pstep.argtypes = [vp]
    lib.pfe_solve.argtypes = [vp, i32, i32, vp, vp, C.POINTER(SolveStats)]
    lib.pfe_destroy.argtypes = [vp]
    lib.pfe_last_error.argtypes = [vp]
    lib.pfe_last_error.restype = C.c_char_p
    lib.pfe_status_string.argtypes = [C.c_int]
    lib.pfe_status_string.restype = C.c_char_p
    lib.pfe_get_info.argtypes = [vp, C.POINTER(Info)]
    lib.pfe_set_stream.argtypes = [vp, vp]
    lib.pfe_get_array.argtypes = [vp, i32, vp]
    lib.pfe_set_array.argtypes = [vp, i32, vp]
    lib.pfe_get_edges.argtypes = [vp, vp, vp, vp]
    lib.pfe_apply_A.argtypes = [vp, vp, vp]
    lib.pfe_solve_system.argtypes = [vp, vp, vp, C.POINTER(StepStats)]
    lib.pfe_time_kernel.argtypes = [vp, i32, i32, C.POINTER(dbl)]
    lib.pfe_fsai_param_count.argtypes = []
    lib.pfe_fsai_set.argtypes = [vp, vp]
    lib.pfe_fsai_classical.argtypes = [vp]
    lib.pfe_fsai_loss_grad.argtypes = [vp, vp, vp, C.POINTER(dbl)]
    lib.pfe_fsai_loss_grad_rhs.argtypes = [vp, vp, vp, i32, dbl, vp, C.POINTER(dbl), C.POINTER(dbl)]
    lib.pfe_fsai_get.argtypes = [vp, vp, vp]
    lib.pfe_adam_update.argtypes = [vp, vp, vp, vp, i64, i32, dbl, dbl, dbl, dbl, vp]
    lib.pfe_get_segments.argtypes = [vp, vp, vp]
    lib.pfe_get_segment_stats.argtypes = [vp, vp, vp, vp]
    lib.pfe_laplacian_eigenmap.argtypes = [vp, i32, vp, i32, dbl, C.POINTER(i32), C.POINTER(dbl)]
    lib.pfe_objective.argtypes = [vp, i32, C.POINTER(dbl), C.POINTER(dbl)]
    lib.pfe_autotune.argtypes = [vp, i32, vp, vp]
    lib.pfe_set_variant.argtypes = [vp, i32, i32]
    lib.pfe_solve_two_stage.argtypes = [vp, i32, i32, i32, vp, vp, C.POINTER(SolveStats)]
    lib.pfe_kmeans.argtypes = [vp, vp, i32, i32, vp, i32, vp, vp, C.POINTER(dbl), C.POINTER(i32)]
    lib.pfe_residual.argtypes = [vp, vp, vp, vp]
    lib.pfe_get_variant.argtypes = [vp, i32, C.POINTER(i32), vp]
    lib.pfe_get_shape.argtypes = [vp, i32, C.POINTER(i32), vp]
    lib.pfe_set_shape.argtypes = [vp, i32, i32]
    for name in EXPORTS:
        if name not in ("pfe_default_params", "pfe_last_error", "pfe_status_string"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class PFEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def _ptr(a, dtype=np.float64):
    """(pointer, keep-alive) for a numpy array or torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected C-contiguous {np.dtype(dtype).name} array")
        return a.ctypes.data, a
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        want = torch.float64 if dtype == np.float64 else torch.int32
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected contiguous {want} tensor")
        return a.data_ptr(), a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class PFE:
    """One embedding problem -- or a batch of independent problems (``shapes``
    for images, ``seg_off`` for edge lists) -- with graph, system matrix and
    iteration state on the GPU."""

    def __init__(self, features, *, sigma: float, H: int | None = None, W: int | None = None,
                 radius: float | None = None, edges=None, lam: float = 0.0, r: float = 1.0,
                 precision: str = "mixed", tol: float = 1e-6, max_iter: int = 5000, refresh: int = 50,
                 reset_inner: bool = True, loop: str = "graph", check_every: int = 4,
                 blocks_per_sm: int = 0, stream=None, shapes=None, seg_off=None, max_device_bytes: int = 0):
        self.lib = load_library()
        self.ctx = C.c_void_p()
        fp, self._feat = _ptr(features)
        n, m = features.shape
        gd = GraphDesc()
        gd.n, gd.m, gd.features, gd.sigma = n, m, fp, float(sigma)
        keep = []
        if edges is None:
            gd.kind, gd.radius = PFE_GRAPH_GRID, float(radius)
            if shapes is not None:  # batch of images: (H_s, W_s) each
                hw = np.ascontiguousarray(np.asarray(shapes, dtype=np.int32).reshape(-1))
                keep.append(hw)
                gd.nseg, gd.seg_hw = len(shapes), hw.ctypes.data
            else:
                gd.H, gd.W = int(H), int(W)
        else:
            ei, ej = edges
            pi, self._ei = _ptr(ei, np.int32)
            pj, self._ej = _ptr(ej, np.int32)
            gd.kind, gd.ei, gd.ej, gd.n_edges = PFE_GRAPH_EDGES, pi, pj, int(ei.shape[0])
            if seg_off is not None:
                so = np.ascontiguousarray(np.asarray(seg_off, dtype=np.int64))
                keep.append(so)
                gd.nseg, gd.seg_off = len(so) - 1, so.ctypes.data
        p = Params()
        self.lib.pfe_default_params(C.byref(p))
        p.lambda_, p.r = float(lam), float(r)
        p.precision = PFE_MIXED if precision == "mixed" else PFE_FP64
        p.tol, p.max_iter, p.refresh = float(tol), int(max_iter), int(refresh)
        p.reset_inner_each_outer = 1 if reset_inner else 0
        p.loop_mode = PFE_LOOP_GRAPH if loop == "graph" else PFE_LOOP_HOST
        p.check_every, p.blocks_per_sm = int(check_every), int(blocks_per_sm)
        p.max_device_bytes = int(max_device_bytes)
        self.params = p
        self.n = n
        self.d = 0
        st = self.lib.pfe_build_graph(C.byref(self.ctx), C.byref(gd), C.byref(p), _stream_ptr(stream))
        self._feat = self._ei = self._ej = None
        if st != PFE_OK:
            raise PFEError(st, f"pfe_build_graph failed: {self.lib.pfe_status_string(st).decode()}: "
                               f"{self.lib.pfe_last_error(None).decode()}")

    # -- helpers
    def _check(self, st: int, what: str, ok=(PFE_OK,)):
        if st not in ok:
            msg = self.lib.pfe_last_error(self.ctx).decode()
            raise PFEError(st, f"{what}: {self.lib.pfe_status_string(st).decode()}: {msg}")
        return st

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            self.lib.pfe_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API
    def info(self) -> dict:
        i = Info()
        self._check(self.lib.pfe_get_info(self.ctx, C.byref(i)), "pfe_get_info")
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def set_stream(self, stream):
        self._check(self.lib.pfe_set_stream(self.ctx, _stream_ptr(stream)), "pfe_set_stream")

    def segments(self):
        """(row offsets [nseg + 1], lambda per segment) of a batch."""
        ns = self.info()["nseg"]
        off = np.empty(ns + 1, dtype=np.int64)
        lam = np.empty(ns, dtype=np.float64)
        self._check(self.lib.pfe_get_segments(self.ctx, off.ctypes.data, lam.ctypes.data), "pfe_get_segments")
        return off, lam

    def segment_stats(self, totals: bool = False):
        """(iterations [nseg], relative residuals [nseg, d]) of the last PCG
        solve; with totals, also each segment's iterations summed over the
        solves of the last solve() call."""
        ns = self.info()["nseg"]
        it = np.empty(ns, dtype=np.int32)
        rr = np.empty((ns, self.d), dtype=np.float64)
        tot = np.empty(ns, dtype=np.int64)
        self._check(self.lib.pfe_get_segment_stats(self.ctx, it.ctypes.data, rr.ctypes.data, tot.ctypes.data),
                    "pfe_get_segment_stats")
        return (it, rr, tot) if totals else (it, rr)

    def init(self, Y0=None, d: int | None = None):
        """Start from Y0 (n x d), or from the Laplacian eigenmap when Y0 is None."""
        if Y0 is None:
            self._check(self.lib.pfe_init(self.ctx, int(d), None, int(d)), "pfe_init")
            self.d = int(d)
            return
        d = Y0.shape[1]
        p, keep = _ptr(Y0)
        self._check(self.lib.pfe_init(self.ctx, d, p, d), "pfe_init")
        self.d = d

    def autotune(self, reps: int = 20):
        """Time the SpMM variants on this problem and keep the fastest:
        (chosen variant, {variant: ms} of those that apply)."""
        choice = np.zeros(1, dtype=np.int32)
        ms = np.zeros(SPMM_NVARIANTS, dtype=np.float64)
        self._check(self.lib.pfe_autotune(self.ctx, int(reps), choice.ctypes.data, ms.ctypes.data), "pfe_autotune")
        return int(choice[0]), {v: float(t) for v, t in enumerate(ms) if t >= 0}

    def set_variant(self, variant: int, kernel: int | str = 0):
        kernel = TUNE.get(kernel, kernel) if isinstance(kernel, str) else kernel
        self._check(self.lib.pfe_set_variant(self.ctx, int(kernel), int(variant)), "pfe_set_variant")

    def get_variant(self, kernel: int | str = 0):
        """(current variant, timings of the column forms from the last autotune
        (the FSAI kernels or the edge pass), or None for the SpMM)."""
        kernel = TUNE.get(kernel, kernel) if isinstance(kernel, str) else kernel
        v = C.c_int32()
        ms = np.full(2, -1.0)
        self._check(self.lib.pfe_get_variant(self.ctx, int(kernel), C.byref(v), ms.ctypes.data), "pfe_get_variant")
        return v.value, (None if kernel == 0 else ms)

    def get_shape(self, kernel: str):
        """(blocks per SM chosen for a row kernel (0: its occupancy), {blocks
        per SM: ms} timed by the last autotune)."""
        b = C.c_int32()
        ms = np.full(8, -1.0)
        self._check(self.lib.pfe_get_shape(self.ctx, KERNEL[kernel], C.byref(b), ms.ctypes.data), "pfe_get_shape")
        return b.value, {k + 1: float(t) for k, t in enumerate(ms) if t > 0}

    def set_shape(self, kernel: str, blocks_per_sm: int):
        self._check(self.lib.pfe_set_shape(self.ctx, KERNEL[kernel], int(blocks_per_sm)), "pfe_set_shape")

    def kmeans(self, k: int, X=None, C0=None, max_iter: int = 100):
        """k-means segmentation of X (n x d) or of the embedding: (labels,
        centroids, inertia, rounds)."""
        d = (self.d or 1) if X is None else X.shape[1]  # before pfe_init the library reports PFE_ESTATE
        px, kx = _ptr(X) if X is not None else (None, None)
        pc, kc = _ptr(C0) if C0 is not None else (None, None)
        labels = np.empty(self.n, dtype=np.int32)
        cent = np.empty((k, d))
        inertia, rounds = C.c_double(), C.c_int32()
        self._check(self.lib.pfe_kmeans(self.ctx, px, int(d), int(k), pc, int(max_iter), labels.ctypes.data,
                                        cent.ctypes.data, C.byref(inertia), C.byref(rounds)), "pfe_kmeans")
        return labels, cent, inertia.value, rounds.value

    def residual(self, B, X):
        """|B - A X| / |B| per problem and column ([nseg, d]) with the FP64 values of A."""
        pb, kb = _ptr(B)
        px, kx = _ptr(X)
        out = np.empty((self.info()["nseg"], X.shape[1]), dtype=np.float64)
        self._check(self.lib.pfe_residual(self.ctx, pb, px, out.ctypes.data), "pfe_residual")
        return out

    def objective(self, which: str = "yhat"):
        """(|M Y|_1, |Y^T D Y - I|_F) of the iterate ("y") or the embedding ("yhat")."""
        l1, oe = C.c_double(), C.c_double()
        self._check(self.lib.pfe_objective(self.ctx, 0 if which == "y" else 1, C.byref(l1), C.byref(oe)),
                    "pfe_objective")
        return l1.value, oe.value

    def laplacian_eigenmap(self, d: int, max_iter: int = 400, tol: float = 1e-9, out=None,
                           allow_notconv: bool = False):
        """(V [n x d], rounds, residual): the Laplacian-eigenmap embedding."""
        V = np.empty((self.n, d)) if out is None else out
        pv, kv = _ptr(V)
        it, res = C.c_int32(), C.c_double()
        ok = (PFE_OK, PFE_ENOTCONV) if allow_notconv else (PFE_OK,)
        self._check(self.lib.pfe_laplacian_eigenmap(self.ctx, int(d), pv, int(max_iter), float(tol), C.byref(it),
                                                    C.byref(res)), "pfe_laplacian_eigenmap", ok)
        return V, it.value, res.value

    def inner_step(self, stats: bool = False, allow_notconv: bool = False):
        if not stats:
            self._check(self.lib.pfe_inner_step(self.ctx, None), "pfe_inner_step")
            return None
        s = StepStats()
        ok = (PFE_OK, PFE_ENOTCONV) if allow_notconv else (PFE_OK,)
        self._check(self.lib.pfe_inner_step(self.ctx, C.byref(s)), "pfe_inner_step", ok)
        return {"pcg_iters": s.pcg_iters, "converged": bool(s.converged), "relres_max": s.relres_max}

    def pstep(self):
        self._check(self.lib.pfe_pstep(self.ctx), "pfe_pstep")

    def solve(self, n_outer: int, n_inner: int, Y_out=None, Yhat_out=None, allow_notconv: bool = False):
        py, ky = _ptr(Y_out)
        ph, kh = _ptr(Yhat_out)
        s = SolveStats()
        ok = (PFE_OK, PFE_ENOTCONV) if allow_notconv else (PFE_OK,)
        st = self._check(self.lib.pfe_solve(self.ctx, n_outer, n_inner, py, ph, C.byref(s)), "pfe_solve", ok)
        return {"pcg_iters_total": s.pcg_iters_total, "pcg_iters_max": s.pcg_iters_max, "n_solves": s.n_solves,
                "n_unconverged": s.n_unconverged, "relres_max": s.relres_max,
                "kernel_launches": s.kernel_launches, "pcg_rounds": s.pcg_rounds,
                "replacements": s.replacements, "status": st}

    def solve_two_stage(self, n_outer: int, n_inner: int, n_stage2: int, Y_out=None, Yhat_out=None,
                        allow_notconv: bool = False):
        """Stage I (n_outer x n_inner with P-steps), then n_stage2 split-Bregman
        iterations with P, B held (Sec. IV)."""
        py, ky = _ptr(Y_out)
        ph, kh = _ptr(Yhat_out)
        s = SolveStats()
        ok = (PFE_OK, PFE_ENOTCONV) if allow_notconv else (PFE_OK,)
        st = self._check(self.lib.pfe_solve_two_stage(self.ctx, n_outer, n_inner, n_stage2, py, ph, C.byref(s)),
                         "pfe_solve_two_stage", ok)
        return {"pcg_iters_total": s.pcg_iters_total, "pcg_iters_max": s.pcg_iters_max, "n_solves": s.n_solves,
                "n_unconverged": s.n_unconverged, "relres_max": s.relres_max,
                "kernel_launches": s.kernel_launches, "pcg_rounds": s.pcg_rounds,
                "replacements": s.replacements, "status": st}

    def get(self, which: str, out=None):
        if out is None:
            rows = self.n
            if which == "BS":
                rows = self.info()["n_edges"]
            shape = (rows,) if which in ("DEG", "DIAG") else (rows, self.d)
            out = np.empty(shape, dtype=np.float64)
        p, keep = _ptr(out)
        self._check(self.lib.pfe_get_array(self.ctx, ARR[which], p), f"pfe_get_array({which})")
        return out

    def set(self, which: str, arr):
        p, keep = _ptr(arr)
        self._check(self.lib.pfe_set_array(self.ctx, ARR[which], p), f"pfe_set_array({which})")

    def edges(self):
        ne = self.info()["n_edges"]
        a = np.empty(ne, dtype=np.int32)
        b = np.empty(ne, dtype=np.int32)
        w = np.empty(ne, dtype=np.float64)
        self._check(self.lib.pfe_get_edges(self.ctx, a.ctypes.data, b.ctypes.data, w.ctypes.data),
                    "pfe_get_edges")
        return a, b, w

    def apply_A(self, X, out=None):
        out = np.empty_like(X) if out is None else out
        px, kx = _ptr(X)
        po, ko = _ptr(out)
        self._check(self.lib.pfe_apply_A(self.ctx, px, po), "pfe_apply_A")
        return out

    def solve_system(self, RHS, Y, allow_notconv: bool = False):
        """Solve A Y = RHS in place (Y holds the initial guess); returns stats."""
        pr, kr = _ptr(RHS)
        py, ky = _ptr(Y)
        s = StepStats()
        ok = (PFE_OK, PFE_ENOTCONV) if allow_notconv else (PFE_OK,)
        self._check(self.lib.pfe_solve_system(self.ctx, pr, py, C.byref(s)), "pfe_solve_system", ok)
        return {"pcg_iters": s.pcg_iters, "converged": bool(s.converged), "relres_max": s.relres_max}

    def time_kernel(self, which: str, reps: int = 20) -> float:
        """Average milliseconds of one launch of a hot-path kernel (CUDA events)."""
        ms = C.c_double()
        self._check(self.lib.pfe_time_kernel(self.ctx, KERNEL[which], int(reps), C.byref(ms)),
                    f"pfe_time_kernel({which})")
        return ms.value

    # -- learned FSAI preconditioner
    def fsai_set(self, params):
        """Build G from the network parameters (None: back to Jacobi)."""
        if params is None:
            self._check(self.lib.pfe_fsai_set(self.ctx, None), "pfe_fsai_set")
            return
        pp, keep = _ptr_f32(params)
        self._check(self.lib.pfe_fsai_set(self.ctx, pp), "pfe_fsai_set")

    def ic0(self):
        """The paper's incomplete-Cholesky preconditioner, IC(0), for later solves."""
        self._check(self.lib.pfe_ic0(self.ctx), "pfe_ic0")

    def fsai_classical(self):
        """Use the classical FSAI factor (per-row dense solves) as preconditioner."""
        self._check(self.lib.pfe_fsai_classical(self.ctx), "pfe_fsai_classical")

    def fsai_loss_grad(self, params, grad=None):
        """Kaporin loss of G(params) and its gradient (returns (loss, grad))."""
        pp, kp = _ptr_f32(params)
        if grad is None:
            grad = np.empty(self.lib.pfe_fsai_param_count(), dtype=np.float32)
        pg, kg = _ptr_f32(grad)
        loss = C.c_double()
        self._check(self.lib.pfe_fsai_loss_grad(self.ctx, pp, pg, C.byref(loss)), "pfe_fsai_loss_grad")
        return loss.value, grad

    def fsai_loss_grad_rhs(self, params, B, mu: float, grad=None):
        """Kaporin loss plus mu times the mean relative residual of G^T G on
        the right-hand sides B (n x m FP64, host or device): (loss, grad, R)."""
        pp, kp = _ptr_f32(params)
        if grad is None:
            grad = np.empty(self.lib.pfe_fsai_param_count(), dtype=np.float32)
        pg, kg = _ptr_f32(grad)
        pb, kb = _ptr(B)
        loss, rt = C.c_double(), C.c_double()
        self._check(self.lib.pfe_fsai_loss_grad_rhs(self.ctx, pp, pb, int(B.shape[1]), float(mu), pg, C.byref(loss),
                                                    C.byref(rt)), "pfe_fsai_loss_grad_rhs")
        return loss.value, grad, rt.value

    def fsai_get(self):
        info = self.info()
        gd = np.empty(info["n"], dtype=np.float64)
        ge = np.empty(info["n_edges"], dtype=np.float64)
        self._check(self.lib.pfe_fsai_get(self.ctx, gd.ctypes.data, ge.ctypes.data), "pfe_fsai_get")
        return gd, ge


def _ptr_f32(a):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected C-contiguous float32 array")
        return a.ctypes.data, a
    import torch
    if a.dtype != torch.float32 or not a.is_contiguous():
        raise TypeError("expected contiguous float32 tensor")
    return a.data_ptr(), a


def fsai_param_count() -> int:
    return load_library().pfe_fsai_param_count()


def adam_update(params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                eps: float = 1e-8, stream=None):
    """One Adam step on device float32 tensors (libpfe kernel)."""
    lib = load_library()
    st = lib.pfe_adam_update(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), params.numel(),
                             int(step), float(lr), float(beta1), float(beta2), float(eps), _stream_ptr(stream))
    if st != PFE_OK:
        raise PFEError(st, "pfe_adam_update failed")
