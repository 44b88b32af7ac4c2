"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/pfe.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1612_06496_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    with open(os.path.join(ROOT, "include", "pfe.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"PFE_API\s+[\w\s\*]*?\b(pfe_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("pfe_build_graph", "pfe_init", "pfe_inner_step", "pfe_solve"):
        assert name in syms
    assert len(syms) >= 16


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_1612_06496_gb300 import EXPORTS
    assert sorted(EXPORTS) == declared_symbols()


def test_default_params_and_status_strings(lib):
    from paper_1612_06496_gb300.pfe import Params, load_library
    L = load_library()
    p = Params()
    L.pfe_default_params(ctypes.byref(p))
    assert p.r == 1.0 and p.tol == 1e-6 and p.max_iter == 5000 and p.refresh == 50
    assert p.reset_inner_each_outer == 1
    assert L.pfe_status_string(4) == b"PFE_ENOTCONV"


def test_null_arguments_rejected_without_gpu(lib):
    """Argument checks run before any CUDA call."""
    from paper_1612_06496_gb300.pfe import GraphDesc, Params, load_library
    L = load_library()
    ctx = ctypes.c_void_p()
    p = Params()
    L.pfe_default_params(ctypes.byref(p))
    g = GraphDesc()
    assert L.pfe_build_graph(ctypes.byref(ctx), None, ctypes.byref(p), None) == 1
    g.n = 1
    assert L.pfe_build_graph(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(p), None) == 1
    g.n, g.m, g.sigma, g.kind = 16, 5, 0.1, 0
    assert L.pfe_build_graph(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(p), None) == 1  # no features
    assert L.pfe_init(None, 3, None, 3) == 1
    assert L.pfe_inner_step(None, None) == 1
    assert L.pfe_solve(None, 1, 1, None, None, None) == 1
    assert L.pfe_destroy(None) == 0


def test_failed_build_leaves_its_message(lib):
    """pfe_last_error(NULL) reports the calling thread's last failed build
    (its context is gone); a later failure replaces it."""
    from paper_1612_06496_gb300.pfe import GraphDesc, Params, load_library
    L = load_library()
    ctx = ctypes.c_void_p()
    p = Params()
    L.pfe_default_params(ctypes.byref(p))
    g = GraphDesc()
    g.n = 1
    assert L.pfe_build_graph(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(p), None) == 1
    assert L.pfe_last_error(None) == b"PFE_EINVAL" and not ctx.value
    g.n, g.m, g.sigma, g.kind, g.features, g.radius, g.H, g.W = 16, 5, 0.1, 0, 8, 2.0, 4, 4
    p.precond = 7  # not a preconditioner the build takes
    assert L.pfe_build_graph(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(p), None) == 8
    assert L.pfe_last_error(None) == b"PFE_EUNSUPPORTED"


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets that
    the C compiler gives the header's struct (gcc compiles a probe of
    sizeof/offsetof; nothing of the library runs)."""
    import shutil
    import subprocess
    from paper_1612_06496_gb300 import pfe as B
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    pairs = {"pfe_graph_desc": B.GraphDesc, "pfe_params": B.Params, "pfe_info": B.Info,
             "pfe_step_stats": B.StepStats, "pfe_solve_stats": B.SolveStats}
    lines, want = [], []
    for cname, cls in pairs.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            field = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("%zu\\n", offsetof({cname}, {field}));')
            want.append(getattr(cls, fname).offset)
    src = tmp_path / "probe.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "pfe.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "probe"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want


def test_default_params_have_no_device_cap(lib):
    from paper_1612_06496_gb300.pfe import Params, load_library
    p = Params()
    p.max_device_bytes = 123
    load_library().pfe_default_params(ctypes.byref(p))
    assert p.max_device_bytes == 0
