"""FP64 CPU oracle for the piecewise-flat-embedding hot path.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline leg use it.  The CUDA library never imports it.
"""
from .pfe_oracle import *  # noqa: F401,F403
