"""SpMM kernel variants and the autotuner: every variant against the oracle,
the tuned choice applied to the solve."""
import numpy as np
import pytest

from oracle import pfe_oracle as O
from synth import CONFIGS
from tests.gpu_common import gpu_problem, oracle_graph, relerr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_spmm_variants_match_oracle(variant):
    spec = CONFIGS["C1"]  # radius 2: 12 slots per row, the fixed-length kernels apply
    p, X, Y0 = gpu_problem(spec, "mixed")
    g = oracle_graph(spec, X)
    p.init(Y0)
    p.set_variant(variant)
    Y = np.empty_like(Y0)
    p.solve(2, 3, Y, None)
    st = O.soc_pfe(g, Y0, 2, 3)
    assert relerr(Y, st.Y) <= 2e-4, variant
    p.close()


def test_autotune_chooses_an_applicable_variant():
    spec = CONFIGS["C1"]
    p, X, Y0 = gpu_problem(spec, "mixed")
    p.init(Y0)
    choice, ms = p.autotune(5)
    assert set(ms) == {0, 1, 2, 3} and all(t > 0 for t in ms.values())
    assert ms[choice] == min(ms.values())
    st = p.solve(1, 2)
    assert st["n_unconverged"] == 0
    p.close()
    # FP64 and edge-list graphs: only the general kernel applies
    q, _, _ = gpu_problem(spec, "fp64")
    q.init(Y0)
    choice, ms = q.autotune(3)
    assert choice == 0 and list(ms) == [0]
    q.close()
