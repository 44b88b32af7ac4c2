"""Seeded synthetic inputs shared by the oracle-side tests and the GPU path.

This package draws random numbers and lays out data points; it holds none of
the embedding method's arithmetic (no graph weights, no solves).  Both the
CPU oracle and the CUDA library receive the arrays it returns.
"""
from .images import (  # noqa: F401
    CONFIGS,
    ImageSpec,
    batch_specs,
    crop_specs,
    features_from_image,
    make_image,
    make_problem,
    random_init,
    voronoi_image,
)
