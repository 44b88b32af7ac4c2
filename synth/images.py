"""Synthetic images shaped like the paper's segmentation workload.

The paper evaluates on natural RGB photographs (Sec. IV: BSDS500 training
images, 481x321).  That dataset is not available here, so every workload is a
seeded piecewise-smooth Voronoi image of the same shape: K random sites, a
random colour per region, optional per-region colour gradients and
sinusoidal texture, plus i.i.d. Gaussian noise.  Data points are pixels with
features (R, G, B, 0.1*x/S, 0.1*y/S), S = max(H, W); pixel (x, y) is vertex
p = y*W + x.

The random draws happen in a fixed order (sites, colours, gradients, texture,
noise) from ``numpy.random.default_rng(seed)`` (PCG64), so the same seed gives
the same image on every machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class ImageSpec:
    """One synthetic image and the embedding problem posed on it."""

    name: str
    H: int
    W: int
    regions: int
    noise: float
    seed: int
    gradient: bool = False
    texture: bool = False
    radius: float = 2.0
    sigma: float = 0.1
    d: int = 3
    n_outer: int = 10
    n_inner: int = 10
    tol: float = 1e-8
    # crop window (x0, y0, w, h) taken from the full image; None = whole image
    crop: tuple | None = None
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        if self.crop is not None:
            return self.crop[2] * self.crop[3]
        return self.H * self.W

    @property
    def shape(self) -> tuple[int, int]:
        if self.crop is not None:
            return self.crop[3], self.crop[2]
        return self.H, self.W


# The five workloads: a small FP64 case, a paper-scale image, a batch of
# uneven images, the learned-preconditioner training/eval set and a large
# image.  Sizes, radii, sigmas, d and iteration counts are those of the
# benchmark definitions; the seeds are fixed here.
CONFIGS: dict[str, ImageSpec] = {
    "C1": ImageSpec("C1", 32, 32, 4, 0.05, seed=1, radius=2.0, sigma=0.1, d=3,
                    n_outer=10, n_inner=10, tol=1e-8),
    "C2": ImageSpec("C2", 321, 481, 8, 0.03, seed=2, gradient=True, radius=3.0,
                    sigma=0.08, d=8, n_outer=20, n_inner=10, tol=1e-6),
    # C3 stands for the whole batch (batch_specs()): the per-problem settings
    # shared by its 64 images; H, W, regions and seed here are those of image 0
    "C3": ImageSpec("C3", 96, 96, 3, 0.03, seed=3000, radius=2.0, sigma=0.1, d=5,
                    n_outer=10, n_inner=10, tol=1e-6),
    "C4": ImageSpec("C4", 321, 481, 8, 0.03, seed=49000, gradient=True, radius=3.0,
                    sigma=0.08, d=8, n_outer=1, n_inner=10, tol=1e-6),
    "C5": ImageSpec("C5", 2048, 2048, 40, 0.03, seed=5, texture=True, radius=2.0,
                    sigma=0.1, d=10, n_outer=10, n_inner=10, tol=1e-6),
}


def voronoi_image(spec: ImageSpec) -> np.ndarray:
    """Return the full (uncropped) H x W x 3 float64 image for ``spec``."""
    H, W, K = spec.H, spec.W, spec.regions
    rng = np.random.default_rng(spec.seed)
    sites = np.stack([rng.uniform(0.0, W, size=K), rng.uniform(0.0, H, size=K)], axis=1)
    colours = rng.uniform(0.0, 1.0, size=(K, 3))
    grads = rng.uniform(-0.25, 0.25, size=(K, 3, 2)) if spec.gradient else None
    if spec.texture:
        theta = rng.uniform(0.0, 2 * np.pi, size=K)
        period = rng.uniform(8.0, 32.0, size=K)
        phase = rng.uniform(0.0, 2 * np.pi, size=K)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    # nearest site; ties go to the lower site index (strict < keeps the first)
    best = np.full((H, W), np.inf)
    label = np.zeros((H, W), dtype=np.int64)
    for k in range(K):
        dist = (xs - sites[k, 0]) ** 2 + (ys - sites[k, 1]) ** 2
        closer = dist < best
        best[closer] = dist[closer]
        label[closer] = k
    img = colours[label]
    S = float(max(H, W))
    if grads is not None:
        rel = np.stack([xs - sites[label, 0], ys - sites[label, 1]], axis=-1) / S
        img = img + np.einsum("hwcj,hwj->hwc", grads[label], rel)
    if spec.texture:
        proj = np.cos(theta[label]) * xs + np.sin(theta[label]) * ys
        tex = 0.05 * np.sin(2 * np.pi * proj / period[label] + phase[label])
        img = img + tex[..., None]
    img = img + rng.normal(0.0, spec.noise, size=(H, W, 3))
    return img


def make_image(spec: ImageSpec) -> np.ndarray:
    """Image for ``spec``, cropped when the spec names a window."""
    img = voronoi_image(spec)
    if spec.crop is not None:
        x0, y0, w, h = spec.crop
        img = img[y0:y0 + h, x0:x0 + w]
    return np.ascontiguousarray(img)


def features_from_image(img: np.ndarray, coord_scale: float = 0.1) -> np.ndarray:
    """Data points x_p = (R, G, B, s*x/S, s*y/S), p = y*W + x, as an n x 5 array."""
    H, W, _ = img.shape
    S = float(max(H, W))
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    feats = np.concatenate(
        [img.reshape(H * W, 3),
         (coord_scale * xs / S).reshape(-1, 1),
         (coord_scale * ys / S).reshape(-1, 1)], axis=1)
    return np.ascontiguousarray(feats)


def random_init(n: int, d: int, seed: int) -> np.ndarray:
    """Seeded standard-normal n x d starting embedding (before D-orthonormalisation)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.standard_normal((n, d))


def make_problem(spec: ImageSpec):
    """(features, Y0) for ``spec``: the inputs both implementations receive."""
    img = make_image(spec)
    X = features_from_image(img)
    Y0 = random_init(X.shape[0], spec.d, spec.seed)
    return X, Y0


def crop_specs(base: ImageSpec, count: int = 4, size: int = 64, seed: int | None = None):
    """Seeded size x size windows of ``base``'s image, each its own problem."""
    rng = np.random.default_rng((base.seed if seed is None else seed) + 104729)
    out = []
    for c in range(count):
        x0 = int(rng.integers(0, base.W - size + 1))
        y0 = int(rng.integers(0, base.H - size + 1))
        out.append(replace(base, name=f"{base.name}crop{c}", crop=(x0, y0, size, size)))
    return out


def batch_specs(count: int = 64, seed0: int = 3000, wmin: int = 96, wmax: int = 481,
                hmin: int = 96, hmax: int = 321, rmin: int = 3, rmax: int = 12,
                d: int = 5) -> list[ImageSpec]:
    """The batched workload: ``count`` images of uneven size, one seed each."""
    specs = []
    for k in range(count):
        seed = seed0 + k
        rng = np.random.default_rng(seed + 15485863)
        W = int(rng.integers(wmin, wmax + 1))
        H = int(rng.integers(hmin, hmax + 1))
        K = int(rng.integers(rmin, rmax + 1))
        specs.append(ImageSpec(f"C3_{k}", H, W, K, 0.03, seed=seed, radius=2.0, sigma=0.1,
                               d=d, n_outer=10, n_inner=10, tol=1e-6))
    return specs
