"""Shared helpers of the GPU tests: build the library once, run the oracle on
the same seeded inputs, relative errors."""
from __future__ import annotations

import functools

import numpy as np

from oracle import pfe_oracle as O
from synth import CONFIGS, ImageSpec, make_problem


def relerr(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@functools.lru_cache(maxsize=None)
def ensure_built() -> str:
    from paper_1612_06496_gb300 import build
    return build.build()


def gpu_problem(spec: ImageSpec, precision: str, **kw):
    ensure_built()
    from paper_1612_06496_gb300 import PFE
    X, Y0 = make_problem(spec)
    H, W = spec.shape
    p = PFE(X, sigma=spec.sigma, H=H, W=W, radius=spec.radius, precision=precision, **kw)
    return p, X, Y0


def oracle_graph(spec: ImageSpec, X):
    H, W = spec.shape
    return O.build_grid_graph(X, H, W, spec.radius, spec.sigma)


@functools.lru_cache(maxsize=None)
def oracle_run(name: str, n_outer: int, n_inner: int, crop: tuple | None = None):
    spec = CONFIGS[name]
    if crop is not None:
        from dataclasses import replace
        spec = replace(spec, crop=crop)
    X, Y0 = make_problem(spec)
    g = oracle_graph(spec, X)
    st = O.soc_pfe(g, Y0, n_outer, n_inner, solver="direct")
    return g, st, O.embedding(g, st)


def small_spec(H=13, W=17, d=5, seed=11, radius=2.0, sigma=0.1, regions=3):
    return ImageSpec("small", H, W, regions, 0.05, seed=seed, radius=radius, sigma=sigma, d=d)
