"""GB300 (sm_103a) implementation of the piecewise-flat-embedding hot path.

The computation lives in ``_lib/libpfe.so`` (CUDA kernels behind the C ABI
declared in ``include/pfe.h``); ``pfe.PFE`` is a thin ctypes binding.
Build the library with ``python -m paper_1612_06496_gb300.build``.
"""
from .pfe import (  # noqa: F401
    ARR,
    EXPORTS,
    LIB_PATH,
    PFE,
    PFEError,
    load_library,
)
