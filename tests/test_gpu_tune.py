"""SpMM kernel variants and the autotuner: every variant against the oracle,
the tuned choice applied to the solve."""
import numpy as np
import pytest

from oracle import pfe_oracle as O
from synth import CONFIGS
from tests.gpu_common import gpu_problem, oracle_graph, relerr, small_spec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7])
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
    assert set(ms) == {0, 1, 2, 3, 4, 5, 6, 7} and all(t > 0 for t in ms.values())
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


@pytest.mark.parametrize("H,W,d,radius", [(23, 20, 3, 2.0), (29, 32, 4, 3.0), (64, 64, 10, 2.0), (7, 132, 10, 3.0),
                                          (41, 100, 10, 2.0), (40, 3, 5, 3.0), (2, 50, 3, 2.0)])
def test_stencil_spmm_equals_fixed_spmm_bitwise(H, W, d, radius):
    """The stencil-form SpMM (a ring of row bands of p and the rows' matrix
    values staged by bulk copies; no column array) and the fixed-length
    kernels with the columns computed from the stencil add the same products
    in the same order as the fixed-length kernels that read the columns:
    whole solves agree bit for bit (odd d: a left pad for 16-byte alignment;
    d = 4: four columns a lane; a 7-row image: bands clipped at both ends;
    W = 100: a narrower last strip; W = 3 at radius 3 and a 2-row image:
    stencil offsets that leave the image on both sides)."""
    spec = small_spec(H=H, W=W, d=d, radius=radius)
    out = {}
    for variant in (1, 5, 6, 2, 7):
        if variant == 5 and W % 4 != 0:  # the stencil form needs 16-byte aligned image rows
            continue
        p, X, Y0 = gpu_problem(spec, "mixed")
        p.init(Y0)
        p.set_variant(variant)
        Y = np.empty_like(Y0)
        st = p.solve(2, 3, Y, None)
        assert st["n_unconverged"] == 0
        out[variant] = Y
        p.close()
    for v in (5, 6):
        if v in out:
            np.testing.assert_array_equal(out[1], out[v])
    np.testing.assert_array_equal(out[2], out[7])


@pytest.mark.parametrize("H,W,d,radius", [(64, 64, 10, 2.0), (40, 3, 5, 3.0), (33, 47, 8, 3.0), (2, 50, 3, 2.0)])
def test_fsai_stencil_columns_equal_slot_columns_bitwise(H, W, d, radius):
    """The FSAI kernels with the columns computed from the stencil add the
    same products in the same order as with the slot columns: learned-FSAI
    solves agree bit for bit (images narrower and shorter than the stencil
    included)."""
    from paper_1612_06496_gb300.learned import load_weights
    spec = small_spec(H=H, W=W, d=d, radius=radius)
    out = []
    for v in (0, 1):
        p, X, Y0 = gpu_problem(spec, "mixed")
        p.fsai_set(load_weights())
        p.init(Y0)
        p.set_variant(v, "fsai")
        assert p.get_variant("fsai")[0] == v
        Y = np.empty_like(Y0)
        st = p.solve(2, 3, Y, None)
        assert st["n_unconverged"] == 0
        out.append(Y)
        p.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_autotune_picks_the_fsai_column_form():
    """With the learned factor on one grid image the autotuner times both
    column forms of the FSAI kernels and keeps the faster; on a batch only
    the slot columns apply."""
    from paper_1612_06496_gb300 import PFEError
    from paper_1612_06496_gb300.learned import load_weights
    spec = small_spec(H=48, W=52, d=10)
    p, X, Y0 = gpu_problem(spec, "mixed")
    p.fsai_set(load_weights())
    p.init(Y0)
    p.autotune(5)
    v, ms = p.get_variant("fsai")
    assert v in (0, 1) and np.all(ms > 0) and ms[v] == ms.min()
    p.close()
    q, _, Y0 = gpu_problem(spec, "fp64")
    q.init(Y0)
    with pytest.raises(PFEError) as ei:
        q.set_variant(1, "fsai")
    assert ei.value.status == 8
    q.close()


def test_stencil_spmm_needs_aligned_rows():
    """Image rows that do not start on 16-byte boundaries (W % 4 != 0) leave
    the stencil SpMM out: choosing it is PFE_EUNSUPPORTED, the autotuner
    skips it."""
    from paper_1612_06496_gb300 import PFEError
    spec = small_spec(H=16, W=18, d=5)
    p, X, Y0 = gpu_problem(spec, "mixed")
    p.init(Y0)
    with pytest.raises(PFEError) as ei:
        p.set_variant(5)
    assert ei.value.status == 8
    choice, ms = p.autotune(3)
    assert 5 not in ms and choice != 5
    p.close()


@pytest.mark.parametrize("H,W,d", [(64, 64, 10), (41, 100, 10), (2, 50, 3), (40, 3, 5), (19, 530, 4), (23, 29, 7)])
def test_edge_pass_from_the_stencil_equals_slot_arrays_bitwise(H, W, d):
    """The edge pass with each slot's neighbour and its edge's Bregman slot
    computed from the stencil (no column or edge-id array read) forms the
    same products in the same order as with the slot arrays: three inner
    steps give bit-identical Y, b and right-hand sides (an image shorter and
    one narrower than the stencil, ragged widths, odd d)."""
    spec = small_spec(H=H, W=W, d=d)
    out = []
    for v in (0, 1):
        p, X, Y0 = gpu_problem(spec, "mixed")
        p.init(Y0)
        p.set_variant(v, "edge")
        assert p.get_variant("edge")[0] == v
        for _ in range(3):
            p.inner_step()
        out.append((p.get("Y"), p.get("BS"), p.get("RHS")))
        p.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


def test_edge_column_form_applies_to_one_fp32_radius2_image():
    """The stencil form of the edge pass needs one FP32 grid image of radius
    2 (12 slots a row): elsewhere choosing it is PFE_EUNSUPPORTED and the
    autotuner keeps the slot arrays; there it times both and keeps the
    faster."""
    from paper_1612_06496_gb300 import PFEError
    for precision, radius in (("fp64", 2.0), ("mixed", 3.0)):
        spec = small_spec(H=20, W=24, d=4, radius=radius)
        p, X, Y0 = gpu_problem(spec, precision)
        p.init(Y0)
        with pytest.raises(PFEError) as ei:
            p.set_variant(1, "edge")
        assert ei.value.status == 8
        p.autotune(3)
        assert p.get_variant("edge")[0] == 0
        p.close()
    spec = small_spec(H=40, W=44, d=6)
    p, X, Y0 = gpu_problem(spec, "mixed")
    p.init(Y0)
    p.autotune(3)
    v, ms = p.get_variant("edge")
    assert v in (0, 1) and np.all(ms > 0) and ms[v] == ms.min()
    p.close()


def test_timing_the_edge_pass_leaves_the_iteration_state():
    """Timing the edge pass (pfe_time_kernel, and the autotuner's edge-form
    choice) right after pfe_init writes neither the first solve's
    right-hand side nor b: the solve that follows is bit for bit the one
    without the timing."""
    spec = small_spec(H=30, W=34, d=6)
    out = []
    for timed in (False, True):
        p, X, Y0 = gpu_problem(spec, "mixed")
        p.init(Y0)
        if timed:
            p.time_kernel("edge", 3)
            p.set_variant(1, "edge")
            p.time_kernel("edge", 3)
            p.set_variant(0, "edge")
        Y = np.empty_like(Y0)
        p.solve(1, 3, Y, None)
        out.append(Y)
        p.close()
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("precond", ["jacobi", "learned"])
def test_autotuned_launch_shapes(precond):
    """pfe_autotune also chooses the blocks per SM of each row kernel the
    iteration runs (the SpMM, k_update and k_pupdate or k_fsai_tr and
    k_fsai_zp, the edge pass): the default (occupancy) is timed with up to
    three smaller counts.  Every shape solves within the FP32 path's 2e-4 of
    the oracle, and a shape's solve is reproducible bit for bit; other
    kernels and counts outside 0..8 are refused."""
    from paper_1612_06496_gb300 import PFEError
    from paper_1612_06496_gb300.learned import load_weights
    spec = small_spec(H=96, W=90, d=6)
    kernels = ["spmm", "edge"] + (["fsai_tr", "fsai_zp"] if precond == "learned" else ["update", "pupdate"])

    def problem():
        p, X, Y0 = gpu_problem(spec, "mixed")
        if precond == "learned":
            p.fsai_set(load_weights())
        p.init(Y0)
        return p, X, Y0

    p, X, Y0 = problem()
    p.autotune(3)
    shapes = {k: p.get_shape(k) for k in kernels}
    for k, (b, ms) in shapes.items():
        assert 0 <= b <= 8 and len(ms) >= 1 and all(t > 0 for t in ms.values()), (k, b, ms)
        assert b == 0 or b in ms, (k, b, ms)
    with pytest.raises(PFEError):
        p.get_shape("xflush")
    with pytest.raises(PFEError):
        p.set_shape("spmm", 9)
    p.close()
    g = oracle_graph(spec, X)
    ref = O.soc_pfe(g, Y0, 2, 3, solver="direct").Y
    for k in kernels:
        for b in sorted(shapes[k][1])[:2]:
            out = []
            for _ in range(2):
                p, _, _ = problem()
                p.set_shape(k, b)
                assert p.get_shape(k)[0] == b
                Y = np.empty_like(Y0)
                st = p.solve(2, 3, Y, None)
                assert st["n_unconverged"] == 0
                out.append(Y)
                p.close()
            np.testing.assert_array_equal(out[0], out[1])
            assert relerr(out[0], ref) <= 2e-4, (k, b, relerr(out[0], ref))


def test_shape_of_the_stencil_spmm_is_its_own():
    """With the stencil-form SpMM in use (it sizes its own grid) the SpMM's
    launch shape reads as the default with nothing timed, and setting one is
    PFE_EUNSUPPORTED."""
    from paper_1612_06496_gb300 import PFEError
    spec = small_spec(H=40, W=44, d=6)
    p, X, Y0 = gpu_problem(spec, "mixed")
    p.init(Y0)
    p.set_variant(5)
    assert p.get_shape("spmm") == (0, {})
    with pytest.raises(PFEError) as ei:
        p.set_shape("spmm", 3)
    assert ei.value.status == 8
    p.close()
