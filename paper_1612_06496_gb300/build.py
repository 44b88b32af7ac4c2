"""Compile libpfe.so (the CUDA kernels and the C ABI) for sm_103a, in-tree.

Each translation unit is compiled by its own nvcc process in parallel, then
linked into ``paper_1612_06496_gb300/_lib/libpfe.so``.  Object files are
reused when their source and headers are older than the object.

    python -m paper_1612_06496_gb300.build [--force] [-j N]
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libpfe.so")

SOURCES = ["api.cu", "graph.cu", "pcg.cu", "edge.cu", "pstep.cu", "convert.cu", "fsai.cu", "noalloc.cu", "le.cu", "diag.cu", "kmeans.cu"]
# Template instantiations (precision x groups of d), one generated
# translation unit each, so that nvcc runs them in parallel.  The d values
# must match PFE_DISPATCH_D in csrc/dispatch.cuh.
D_GROUPS = {
    "pcg": [[1, 2, 3, 4], [5, 6, 7, 8], [9, 10, 11, 12], [13, 14, 15, 16], [20], [24], [25], [32]],
    "pstep": [[1, 2, 3, 4, 5, 6, 7, 8], [9, 10, 11, 12, 13, 14, 15, 16], [20, 24], [25, 32]],
    "edge": [[1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 20, 24, 25, 32]],
    # Laplacian-eigenmap block widths (FP64 only)
    "le": [[1, 2, 3, 4, 5, 6, 7, 8, 9, 10], [11, 12, 13, 14, 15, 16], [20, 24, 25, 32]],
}
TYPES = {"le": ("double",)}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _generated_sources() -> list[str]:
    gen = os.path.join(BUILD_DIR, "gen")
    os.makedirs(gen, exist_ok=True)
    out = []
    for comp, groups in D_GROUPS.items():
        for t in TYPES.get(comp, ("float", "double")):
            for gi, ds in enumerate(groups):
                path = os.path.join(gen, f"{comp}_{t}_{gi}.cu")
                text = f'#include "{comp}_kernels.cuh"\n' + "".join(
                    f"PFE_INSTANTIATE({t}, {d})\n" for d in ds)
                if not os.path.exists(path) or open(path).read() != text:
                    with open(path, "w") as f:
                        f.write(text)
                out.append(path)
    return out


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "pfe.h"))
    return hs


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src, *_headers(), __file__])


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                    "-I", os.path.join(ROOT, "include"), "-I", CSRC, "--expt-relaxed-constexpr"]
    if os.environ.get("PFE_PTXAS_V"):
        flags += ["-Xptxas", "-v"]

    def compile_one(src: str):
        obj = os.path.join(BUILD_DIR, os.path.basename(src).replace(".cu", ".o"))
        if not force and not _stale(obj, src):
            return obj, None
        cmd = [cc, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            return obj, f"{' '.join(cmd)}\n{r.stdout}\n{r.stderr}"
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj, None

    srcs = [os.path.join(CSRC, f) for f in SOURCES] + _generated_sources()
    # longest first: the instantiation units dominate
    srcs.sort(key=lambda p: ("_kernels" not in open(p).read(), p))
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    errors = [e for _, e in results if e]
    if errors:
        raise RuntimeError("libpfe build failed:\n" + "\n".join(errors))
    objs = [o for o, _ in results]
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared",
               "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"libpfe link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-j", type=int, default=None)
    ap.add_argument("-v", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, jobs=a.j, verbose=a.v))
