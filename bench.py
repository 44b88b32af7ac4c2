#!/usr/bin/env python
"""Benchmark of the piecewise-flat-embedding hot path on one GB300.

Metric: seconds per outer iteration (one SOC iteration of Alg. 1 = n_inner
split-Bregman iterations of Alg. 2, each a d-column PCG solve of Eq. 13 to
relative residual 1e-6 plus the fused edge pass, then the P/B-step), with
the PCG iteration counts, for the FP32 path (FP32 edge/SpMM/vectors,
double-FP32 dots and solution, FP64 P-step) next to the plain FP64 path.

Workload (default): the 2048x2048 synthetic image (40 Voronoi regions with
texture, noise 0.03), radius-2 graph (n = 4,194,304, 50,290,692 directed
edges), sigma = 0.1, d = 10, 10 inner iterations per outer iteration.  A
step is one outer iteration, continuing the same solve; the working set of
a step (several GB) is far larger than L2, so no flush is needed between
steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank solves its own image (seed + rank): independent
replicas, weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PFE sec/outer-iter & PCG iters @1e-6 res, learned+FP32 vs plain FP64"
UNIT = "s/outer-iter"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="C5", choices=["C1", "C2", "C3", "C5"],
                    help="C3 is the batch of 64 uneven images (one problem per image, iterated together)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--precond", default="learned", choices=["learned", "jacobi", "classical", "ic0"],
                    help="preconditioner of the timed FP32 arm (learned FSAI, Jacobi, classical FSAI or "
                         "the paper's incomplete Cholesky IC(0))")
    ap.add_argument("--no-alt", action="store_true", help="skip the FP32 arm with the other preconditioner")
    ap.add_argument("--alt-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-worker", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-window", type=int, default=192)
    ap.add_argument("--size", type=int, default=0,
                    help="square image side overriding the workload's size (profiling runs on a smaller case)")
    ap.add_argument("--n-inner", type=int, default=0, help="override inner iterations per outer step")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="PCG loop driver; 'host' launches every kernel from the host (for ncu launch lists)")
    return ap.parse_args()


# --------------------------------------------------------------------------
# CPU oracle sample (runs in a fresh single-threaded process)
# --------------------------------------------------------------------------


def cpu_sample_worker(arg: str):
    """One outer iteration per step of the oracle (Jacobi-PCG mode, or with
    "solver": "direct" its sparse-LU mode, A factored once before the steps),
    single threaded, on one window of the workload's image with the full
    image's lambda (or, for the batch, on one of its images); prints JSON."""
    import numpy as np

    from oracle import pfe_oracle as O
    from synth import CONFIGS, make_problem
    from dataclasses import replace
    cfg = json.loads(arg)
    if cfg["workload"] == "C3":
        from synth import batch_specs
        specs = sorted(batch_specs(), key=lambda s: s.n)
        spec = specs[cfg["index"] % len(specs)]  # the smallest images first, each with its own lambda
        X, Y0 = make_problem(spec)
        g = O.build_grid_graph(X, spec.H, spec.W, spec.radius, spec.sigma)
    else:
        spec = CONFIGS[cfg["workload"]]
        x0, y0, win_w, win_h = cfg["window"]
        wspec = replace(spec, crop=(x0, y0, win_w, win_h))
        X, Y0 = make_problem(wspec)
        g = O.build_grid_graph(X, win_h, win_w, spec.radius, spec.sigma, lam=cfg["lambda"])
    st = O.init_state(g, Y0)
    factor_s = 0.0
    if cfg.get("solver", "pcg") == "direct":
        t0 = time.perf_counter()
        solve = O.DirectSolver(g.A)
        factor_s = time.perf_counter() - t0
    else:
        solve = O.PCGSolver(g.A, spec.tol, 5000, 50)
    times, iters = [], []
    for _ in range(cfg["steps"]):
        t0 = time.perf_counter()
        O.reset_inner(st)
        its = 0
        for _ in range(spec.n_inner):
            info = O.split_bregman_step(g, st, solve)
            its += int(info["iters"].max())
        O.p_and_b_step(g, st)
        times.append(time.perf_counter() - t0)
        iters.append(its / spec.n_inner)
    nnz = g.A.nnz
    print(json.dumps({"times": times, "iters": iters, "nnz": int(nnz), "n": int(g.n), "factor_s": factor_s}))


def cpu_windows(spec, window: int, count: int) -> list:
    """`count` windows of window x window pixels (the whole image when it is
    smaller) spread over the image on a regular grid, distinct when they fit."""
    ww, wh = min(window, spec.W), min(window, spec.H)
    k = 1
    while k * k < count:
        k += 1
    out = []
    for q in range(count):
        gx, gy = q % k, q // k
        x0 = ((spec.W - ww) * (2 * gx + 1)) // (2 * k)
        y0 = ((spec.H - wh) * (2 * gy + 1)) // (2 * k)
        out.append((x0, y0, ww, wh))
    return out


def cpu_cores() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def run_cpu_sample(workload: str, lam: float, steps: int, window: int, nnz_full: int, solver: str = "pcg") -> dict:
    """The oracle, as it stands and single threaded, on one window (the batch:
    one image) per host core, all at once: the seconds a step of the
    slowest one took, times nnz_A of the whole workload over the nnz_A the
    cores processed together, estimates the seconds per outer iteration of
    the whole workload on these cores."""
    from synth import CONFIGS
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    spec = CONFIGS[workload]
    whole = workload != "C3" and window >= spec.W and window >= spec.H
    cores = 1 if whole else cpu_cores()  # an image that fits one window runs whole, on one core
    wins = cpu_windows(spec, window, cores) if workload != "C3" else [None] * cores
    procs = []
    for q in range(cores):
        arg = json.dumps({"workload": workload, "lambda": lam, "steps": steps, "window": wins[q], "index": q,
                          "solver": solver})
        procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-sample-worker", arg],
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT))
    outs = []
    for pr in procs:
        so, se = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("CPU oracle sample failed:\n" + se[-2000:])
        outs.append(json.loads(so.strip().splitlines()[-1]))
    nnz_done = sum(o["nnz"] for o in outs)
    scale = nnz_full / nnz_done
    per_step = [max(o["times"][k] for o in outs) for k in range(steps)]
    return {"times": per_step, "iters": [sum(o["iters"][k] for o in outs) / cores for k in range(steps)],
            "nnz": nnz_done, "n": sum(o["n"] for o in outs), "scale": scale, "cores": cores,
            "window": wins[0][2:] if wins[0] else None, "per_step_scaled": [t * scale for t in per_step],
            "factor_s": max(o.get("factor_s", 0.0) for o in outs)}


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)  # every line the sampler printed
        return self.summarise(self.lines)

    @staticmethod
    def summarise(lines) -> dict | None:
        """Median and largest SM clock over the samples of FIELDS, and every
        throttle reason that was active in any of them."""
        sms, maxs, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxs = max(maxs, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return None
        sms.sort()
        return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": maxs, "reasons": sorted(reasons),
                "samples": len(sms)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("pcg_kernels.cuh", "common.cuh", "tma.cuh"):
        with open(os.path.join(ROOT, "paper_1612_06496_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, kernel: str, units_full: float, variant: int | None = None) -> float | None:
    """DRAM bytes per launch from the committed ncu summary, scaled to the
    full launch; None when the kernel source changed since the capture or
    the capture was of another kernel variant than the one timed."""
    name = f"{kernel}_v{variant}" if variant is not None else kernel  # SpMM: one file per variant
    path = os.path.join(ROOT, "profiles", f"{name}_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as f:
        for ln in f:
            if "=" in ln and not ln.startswith("#"):
                k, v = ln.split("=", 1)
                kv[k.strip()] = v.strip()
    if kv.get("kernel_sha") != kernel_source_hash():
        return None
    if variant is not None and "variant" in kv and kv["variant"] != str(variant):
        return None
    try:
        return float(kv["dram_bytes_per_launch"]) * units_full / float(kv["units"])
    except (KeyError, ValueError):
        return None


# --------------------------------------------------------------------------
# reference arm: the FP64 oracle, timed as it stands on the host cores
# --------------------------------------------------------------------------


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    from synth import CONFIGS, make_problem
    from oracle import pfe_oracle as O
    spec = CONFIGS[args.workload]
    # lambda of the full image, and its nnz_A, for the scale of the sample
    nnz_full, lam = full_graph_size_and_lambda(spec)
    steps = args.warmup + args.steps
    out = run_cpu_sample(args.workload, lam, steps, args.cpu_window, nnz_full)
    timed = out["per_step_scaled"][args.warmup:]
    v = sum(timed) / len(timed)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(spec, args.gpus),
        "pcg_iters_mean": sum(out["iters"][args.warmup:]) / len(timed),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": out["cores"], "kind": "oracle",
                         "sample": cpu_sample_text(spec, args.cpu_window, out)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_sample_text(spec, window: int, out: dict) -> str:
    pcg = f"oracle (FP64, Jacobi-PCG tol {spec.tol:g}, single threaded per process)"
    if spec.name == "C3":
        return (f"{pcg}, one outer iteration per step on {out['cores']} images of the batch at once (the smallest, "
                f"each with its own lambda; {out['iters'][0]:.0f} PCG iterations per solve on average), extrapolated "
                f"to the whole batch by nnz_A ({out['scale']:.1f}x the nonzeros the {out['cores']} cores processed)")
    if out["scale"] <= 1.0 + 1e-12:
        return (f"{pcg}, one outer iteration per step on the whole image ({out['iters'][0]:.0f} PCG iterations "
                f"per solve)")
    w, h = out["window"]
    return (f"{pcg}, one outer iteration per step on {out['cores']} {w}x{h} windows of the same image at once (one "
            f"per host core, spread over the image, the full image's lambda; {out['iters'][0]:.0f} PCG iterations "
            f"per solve on average); the slowest window's time extrapolated to the whole image by nnz_A "
            f"({out['scale']:.1f}x the nonzeros the {out['cores']} cores processed)")


def problem_inputs(spec, rank: int, world: int):
    """(features, Y0, geometry kwargs of PFE, spec of the first problem) of the
    workload; the batch stacks its images' rows (replicas: other seeds)."""
    import numpy as np
    from synth import batch_specs, make_problem
    if spec.name == "C3":
        specs = batch_specs(seed0=3000 + 64 * rank) if world > 1 else batch_specs()
        probs = [make_problem(s) for s in specs]
        X = np.ascontiguousarray(np.vstack([p[0] for p in probs]))
        Y0 = np.ascontiguousarray(np.vstack([p[1] for p in probs]))
        return X, Y0, {"shapes": [s.shape for s in specs]}, specs[0]
    spec = replica_spec(spec, rank, world)
    X, Y0 = make_problem(spec)
    H, W = spec.shape
    return X, Y0, {"H": H, "W": W}, spec


def replica_spec(spec, rank: int, world: int):
    """Each rank solves its own image: the workload with seed + rank."""
    from dataclasses import replace
    return replace(spec, seed=spec.seed + rank) if world > 1 else spec


def max_over_ranks_dist(v: float, world: int, device: str) -> float:
    """The slowest rank's value (the job's time), over torch.distributed."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_outer(ms_max: float, steps: int, world: int) -> float:
    """Whole-job seconds per outer iteration: world replicas each ran `steps`
    outer iterations inside the slowest rank's ms_max."""
    return ms_max / 1e3 / (steps * world)


def full_graph_size_and_lambda(spec):
    """nnz_A and lambda = sqrt(vol) of the full image (the batch: total nnz_A,
    lambda unused), from the oracle's graph definition (pure NumPy; no GPU)."""
    import numpy as np
    from oracle import pfe_oracle as O
    from synth import make_problem
    if spec.name == "C3":
        from synth import batch_specs
        tot = 0
        for s in batch_specs():
            a, _ = O.grid_edges(s.H, s.W, s.radius)
            tot += s.n + 2 * a.shape[0]
        return tot, 0.0
    X, _ = make_problem(spec)
    a, b = O.grid_edges(spec.H, spec.W, spec.radius)
    w = O.heat_kernel_weights(X, a, b, spec.sigma)
    vol = 2.0 * float(np.sum(w))
    return spec.n + 2 * a.shape[0], float(np.sqrt(vol))


L2_BYTES = 129 * 2 ** 20  # GB300 L2


def stencil_size(radius: float) -> int:
    """Neighbours of an interior pixel: offsets (dx, dy) != 0 with dx^2 + dy^2 <= radius^2."""
    r = int(radius)
    return sum(1 for dy in range(-r, r + 1) for dx in range(-r, r + 1)
               if (dx or dy) and dx * dx + dy * dy <= radius * radius)


def l2_note(n: int, d: int, radius: float) -> str:
    """Whether the PCG loop's data (FP32 matrix value + column per stored
    nonzero, about eight n x d FP32 vectors) outgrows the L2 between timed
    iterations; no flush is done either way."""
    ws = 8 * n * (1 + stencil_size(radius)) + 32 * n * d
    if ws > L2_BYTES:
        return f"PCG working set ~{ws / 2 ** 20:.0f} MiB > {L2_BYTES >> 20} MiB L2: inputs larger than L2, no flush"
    return (f"PCG working set ~{ws / 2 ** 20:.0f} MiB fits in the {L2_BYTES >> 20} MiB L2: no flush, so this "
            f"workload's figures are L2-warm, not HBM-bound")


def workload_config(spec, gpus: int) -> dict:
    if spec.name == "C3":
        from synth import batch_specs
        specs = batch_specs()
        n = sum(s.n for s in specs)
        return {"workload": f"C3: batch of {len(specs)} synthetic Voronoi images, 96..481 x 96..321 pixels, "
                            f"3-12 regions, radius-2 graphs, sigma=0.1, d=5, 10 inner iterations per outer step "
                            f"(every image), PCG rel-res 1e-06, one launch per kernel for the whole batch",
                "n": n, "images": len(specs), "d": 5, "n_inner": 10, "tol": 1e-6,
                "l2": l2_note(n, 5, specs[0].radius),
                "parallelism": f"replicas x{gpus}" if gpus > 1 else "single GPU"}
    return {"workload": f"{spec.name}: {spec.W}x{spec.H} synthetic Voronoi image, radius-{spec.radius:g} graph, "
                        f"sigma={spec.sigma:g}, d={spec.d}, {spec.n_inner} inner iterations per outer step, "
                        f"PCG rel-res {spec.tol:g}",
            "n": spec.n, "d": spec.d, "n_inner": spec.n_inner, "tol": spec.tol,
            "l2": l2_note(spec.n, spec.d, spec.radius),
            "parallelism": f"replicas x{gpus}" if gpus > 1 else "single GPU"}


# --------------------------------------------------------------------------
# GB300 arm
# --------------------------------------------------------------------------


def main():
    args = parse()
    if args.cpu_sample_worker is not None:
        cpu_sample_worker(args.cpu_sample_worker)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1612_06496_gb300 import PFE, load_library
    from paper_1612_06496_gb300.learned import load_weights
    from synth import CONFIGS, make_problem
    from dataclasses import replace

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    load_library()
    batch = args.workload == "C3"
    spec = CONFIGS[args.workload]
    if args.size and not batch:
        spec = replace(spec, H=args.size, W=args.size, name=f"{spec.name}@{args.size}")
    X, Y0, geom, spec0 = problem_inputs(spec, rank, world)
    if not batch:
        spec = spec0
    if args.n_inner:
        spec = replace(spec, n_inner=args.n_inner)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        return max_over_ranks_dist(v, world, "cuda")

    Xd = torch.from_numpy(X).cuda()
    Y0d = torch.from_numpy(Y0).cuda()

    tuned = {}
    shapes = {}  # launch shapes chosen by the autotuner, per arm

    def run_arm(precision: str, warmup: int, steps: int, clocks: bool, precond: str = "jacobi"):
        t0 = time.perf_counter()
        p = PFE(Xd, sigma=spec.sigma, radius=spec.radius, precision=precision, tol=spec.tol,
                stream=stream, loop=args.loop, **geom)
        if precond == "learned":
            p.fsai_set(fsai_params)  # network inference of G runs inside the timed setup
        elif precond == "classical":
            p.fsai_classical()
        elif precond == "ic0":
            p.ic0()
        p.init(Y0d)
        # kernel variants (setup): SpMM, FSAI column form, edge-pass column form
        tuned[precision + "/" + precond] = p.autotune(10) + p.get_variant("fsai") + p.get_variant("edge")
        shapes[precision + "/" + precond] = {
            k: p.get_shape(k) for k in ["spmm", "edge"] + (
                ["fsai_tr", "fsai_zp"] if precond in ("learned", "classical") else
                ["update", "pupdate"] if precond == "jacobi" else [])}
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        for _ in range(warmup):
            p.solve(1, spec.n_inner)
        sampler = ClockSampler(local) if clocks else None
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = []
        for _ in range(steps):
            stats.append(p.solve(1, spec.n_inner))
            if batch:  # each image's iterations of this step (64 integers)
                stats[-1]["seg_iters"] = p.segment_stats(totals=True)[2]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        clk = sampler.stop() if sampler else None
        return p, ms, stats, setup_s, clk

    fsai_params = load_weights() if (args.precond == "learned" or not args.no_alt) else None

    # --- FP32 path (the timed arm)
    p, ms, stats, setup_s, clk = run_arm("mixed", args.warmup, args.steps, True, args.precond)
    ms_max = max_over_ranks(ms)
    info = p.info()
    iters_total = sum(s["pcg_iters_total"] for s in stats)
    rounds = sum(s["pcg_rounds"] for s in stats)  # k_spmm launches (a batch: its longest image's iterations)
    n_solves = sum(s["n_solves"] for s in stats)
    if batch:
        # nonzeros x iterations of each image: A_s has n_s + 2|E_s| nonzeros
        import numpy as np
        off, _ = p.segments()
        ea, _, _ = p.edges()
        es = np.bincount(np.searchsorted(off, ea, side="right") - 1, minlength=len(off) - 1)
        nnz_seg = np.diff(off) + 2 * es
        nnz_iters = float(sum(np.dot(nnz_seg, s["seg_iters"]) for s in stats))
    else:
        nnz_iters = float(info["nnz_A"]) * iters_total
    launches = sum(s["kernel_launches"] for s in stats)
    sec_per_outer = job_seconds_per_outer(ms_max, args.steps, world)

    # --- roofline of the dominant kernel: k_spmm (q = A p with the p.q dots)
    spmm_ms = p.time_kernel("spmm", 20)
    upd_ms = p.time_kernel("update", 20)
    pup_ms, puph_ms = p.time_kernel("pupdate", 20), p.time_kernel("pupdate_hold", 20)
    edge_ms = p.time_kernel("edge", 10)
    # the kernels of a replacement iteration (every 50 iterations, after a
    # 1e3-fold fall of a residual, and to confirm convergence): the
    # replacement residual, the update flush, and (FSAI) t = G r with the dots
    repl_ms, xfl_ms = p.time_kernel("replace", 10), p.time_kernel("xflush", 10)
    n, d, nnz, ne = info["n"], info["d"], info["nnz_A"], info["n_edges"]
    fsai_k = {}
    fsai_arm = args.precond in ("learned", "classical")  # the FSAI kernels run (any factor G)
    fsai_cols = tuned.get("mixed/" + args.precond, (0, {}, 0, None))[2]  # 1: columns computed from the stencil
    edge_cols = tuned.get("mixed/" + args.precond, (0, {}, 0, None, 0, None))[4]  # 1: edge pass from the stencil
    if fsai_arm:
        # lower (upper) slots: FP32 G value (+ int32 column unless computed
        # from the stencil) each, G_ii per row; t = G r': r, q in, r', t out;
        # z = G^T t with p_new = z + beta p: t and p in, p_new out, and every
        # other iteration y += alpha_prev p_prev + alpha p: p_prev and y (hi,
        # lo) in, y out
        tr_ms = p.time_kernel("fsai_tr", 20)
        zf_ms, zh_ms = p.time_kernel("fsai_zp", 20), p.time_kernel("fsai_zp_hold", 20)
        ft_ms = p.time_kernel("fsai_t", 10)
        slot_b = (2 if fsai_cols == 1 else 4) * (nnz - n)
        tr_b = slot_b + 4 * n + 16 * n * d
        zh_b = slot_b + 4 * n + 12 * n * d
        zf_b = zh_b + 20 * n * d
        # the network's inference (once per image, in the setup): the 64 x 64
        # layer's 2 * 64 * 64 flops per pattern entry on the tensor cores
        mlp = {}
        if args.precond == "learned":
            n_ent = n + ne
            for name, v in (("tcgen05", 1), ("mma_sync", 0)):
                p.set_variant(v, "mlp")
                t_ms = p.time_kernel("mlp", 5)
                mlp[name] = {"ms": round(t_ms, 4),
                             "tensor_TFLOPs": round(2 * 64 * 64 * n_ent / (t_ms * 1e-3) / 1e12, 1)}
            p.set_variant(1, "mlp")
            mlp["entries"] = n_ent
        fsai_k = {"k_fsai_t_ms": round(ft_ms, 5), "mlp_inference": mlp,
                  "k_fsai_tr_ms": round(tr_ms, 5), "k_fsai_tr_GBps": round(tr_b / (tr_ms * 1e-3) / 1e9, 1),
                  "k_fsai_zp_fold_ms": round(zf_ms, 5), "k_fsai_zp_fold_GBps": round(zf_b / (zf_ms * 1e-3) / 1e9, 1),
                  "k_fsai_zp_hold_ms": round(zh_ms, 5), "k_fsai_zp_hold_GBps": round(zh_b / (zh_ms * 1e-3) / 1e9, 1)}
    # the SpMM variant the autotuner chose for this arm
    variant = tuned.get("mixed/" + args.precond, (0, {}))[0]
    kname = {0: "k_spmm", 1: "k_spmm_fixed", 2: "k_spmm_fixed", 3: "k_spmm_fixed", 4: "k_spmm_tma",
             5: "k_spmm_stencil", 6: "k_spmm_fixed (stencil columns)", 7: "k_spmm_fixed (stencil columns)"}.get(variant,
                                                                                                           "k_spmm")
    if variant in (5, 6, 7):
        # stencil form and computed columns: FP32 value of every nonzero (no
        # column index, no row pointer), p in, q out: 4 nnz_A + 2 * 4 n d
        spmm_bytes = 4 * nnz + 2 * 4 * n * d
    else:
        # FP32 values + int32 indices of A, p in, q out: 8 nnz_A + 4 (n + 1) + 2 * 4 n d
        spmm_bytes = 8 * nnz + 4 * (n + 1) + 2 * 4 * n * d
    # k_update: r, q in, r out, D_A^{-1}; k_pupdate: r, p in, p_new out, D_A^{-1},
    # and on folding iterations p_prev and y (hi, lo) in, y out
    upd_b, puph_b = 3 * 4 * n * d + 4 * n, 3 * 4 * n * d + 4 * n
    pup_b = puph_b + 5 * 4 * n * d
    # candidates for the dominant kernel of the PCG iteration: (name, traffic
    # key, ms per launch, algorithmic bytes per launch); one launch each per
    # iteration (k_fsai_zp: folding and holding launches alternate)
    cands = [("%s<float,%d> (SpMM variant %d)" % (kname, d, variant), "spmm", spmm_ms, spmm_bytes)]
    if fsai_arm:
        cols = " (stencil columns)" if fsai_cols == 1 else ""
        cands += [("k_fsai_tr<float,%d>%s" % (d, cols), "fsai_tr", tr_ms, tr_b),
                  ("k_fsai_zp<float,%d>%s (folding and holding launches averaged)" % (d, cols), "fsai_zp",
                   0.5 * (zf_ms + zh_ms), 0.5 * (zf_b + zh_b))]
    elif args.precond == "jacobi":
        cands += [("k_update<float,%d>" % d, "update", upd_ms, upd_b),
                  ("k_pupdate<float,%d> (folding and holding launches averaged)" % d, "pupdate",
                   0.5 * (pup_ms + puph_ms), 0.5 * (pup_b + puph_b))]
    dom_name, dom_key, dom_ms, dom_bytes = max(cands, key=lambda c: c[2])
    peaks = measured_peaks()
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": round(achieved, 1),
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "peak_source": peaks["source"] + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": ncu_traffic(args.workload, dom_key, nnz,
                                       variant if dom_key == "spmm" else (fsai_cols if fsai_arm else None)),
                "algorithmic_bytes_per_launch": int(dom_bytes), "avg_launch_ms": round(dom_ms, 5),
                "launches_in_timed_region": rounds,
                "share_of_timed_region": round(rounds * dom_ms / ms, 4),
                "spmm": {"kernel": cands[0][0], "ms": round(spmm_ms, 5), "algorithmic_bytes": spmm_bytes,
                         "GBps": round(spmm_bytes / (spmm_ms * 1e-3) / 1e9, 1),
                         "share_of_timed_region": round(rounds * spmm_ms / ms, 4),
                         "traffic": ncu_traffic(args.workload, "spmm", nnz, variant)},
                "other_kernels": {"k_update_ms": round(upd_ms, 5),
                                  "k_update_GBps": round(upd_b / (upd_ms * 1e-3) / 1e9, 1),
                                  "k_pupdate_fold_ms": round(pup_ms, 5),
                                  "k_pupdate_fold_GBps": round(pup_b / (pup_ms * 1e-3) / 1e9, 1),
                                  "k_pupdate_hold_ms": round(puph_ms, 5),
                                  "k_pupdate_hold_GBps": round(puph_b / (puph_ms * 1e-3) / 1e9, 1),
                                  "k_edge_ms": round(edge_ms, 5),
                                  # b read + written (FP32), w, column + edge id per directed slot (none
                                  # when computed from the stencil), Y, C in, RHS out
                                  "k_edge_columns": "stencil" if edge_cols == 1 else "slots",
                                  "k_edge_GBps": round((8 * d * ne + 4 * ne + (0 if edge_cols == 1 else 8 * 2 * ne)
                                                        + 12 * n * d) / (edge_ms * 1e-3) / 1e9, 1),
                                  "replacement_residual_ms": round(repl_ms, 5), "k_xflush_ms": round(xfl_ms, 5),
                                  **fsai_k}}
    # after the timings: the next system of Eq. 13 solved from its warm start
    # by the same path, and |b - A y| / |b| per column with A in FP64
    # (pfe_residual), the problem's matrix rather than the FP32 rounding the
    # iteration multiplies by
    b_next, y_next = p.get("RHS"), p.get("Y")
    p.solve_system(b_next, y_next)
    true_relres = float(p.residual(b_next, y_next).max())
    p.close()

    # --- the FP32 path with the other preconditioner
    alt = None
    if not args.no_alt:
        other = "jacobi" if args.precond == "learned" else "learned"
        qa, msa, sta, _, _ = run_arm("mixed", 1, args.alt_steps, False, other)
        msa = max_over_ranks(msa)
        ita = sum(s["pcg_iters_total"] for s in sta)
        nsa = sum(s["n_solves"] for s in sta)
        alt = {"precond": other, "sec_per_outer_iter": msa / 1e3 / (args.alt_steps * world),
               "pcg_iters_mean": ita / max(nsa, 1), "pcg_iters_max": max(s["pcg_iters_max"] for s in sta),
               "steps": args.alt_steps}
        qa.close()

    # --- plain FP64 path on the same problem
    fp64 = None
    if not args.no_fp64:
        q, ms64, st64, _, _ = run_arm("fp64", 1, args.fp64_steps, False)
        ms64 = max_over_ranks(ms64)
        it64 = sum(s["pcg_iters_total"] for s in st64)
        ns64 = sum(s["n_solves"] for s in st64)
        spmm64 = q.time_kernel("spmm", 5)
        fp64 = {"sec_per_outer_iter": ms64 / 1e3 / (args.fp64_steps * world),
                "pcg_iters_mean": it64 / max(ns64, 1), "pcg_iters_max": max(s["pcg_iters_max"] for s in st64),
                "spmm_ms": round(spmm64, 4),
                "spmm_bound": "fp64 alu: 2 FLOP per nonzero per column at the measured 1.2 TFLOP/s DFMA rate"}
        q.close()

    # --- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        Y0h = torch.from_numpy(Y0).pin_memory()
        Yo = torch.empty(tuple(Y0.shape), dtype=torch.float64).pin_memory()
        Yho = torch.empty_like(Yo).pin_memory()
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            r = PFE(Xh, sigma=spec.sigma, radius=spec.radius, precision="mixed", tol=spec.tol,
                    stream=stream, **geom)
            if args.precond == "learned":
                r.fsai_set(fsai_params)  # host copy of the network weights
            elif args.precond == "classical":
                r.fsai_classical()
            elif args.precond == "ic0":
                r.ic0()
            r.init(Y0h)
            r.solve(1, spec.n_inner, Yo, Yho)
            r.close()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        barrier()
        ms_e2e = max_over_ranks(max(e0.elapsed_time(e1), wall * 1e3))
        e2e = {"value": ms_e2e / 1e3 / (e2e_steps * world), "unit": UNIT,
               "h2d_bytes_per_step": int(X.nbytes + Y0.nbytes + (fsai_params.nbytes if args.precond == "learned" else 0)),
               "d2h_bytes_per_step": int(2 * Yo.numel() * 8),
               "steps": e2e_steps,
               "what": "per step: pfe_build_graph from host features, the preconditioner set up, pfe_init from host Y0, one outer "
                       "iteration (pfe_solve 1 x n_inner), Y and Yhat copied back to pinned host memory"}

    # --- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            out = run_cpu_sample(args.workload, info["lambda_"], 1, args.cpu_window, nnz)
            cpu = {"value": out["per_step_scaled"][0], "unit": UNIT, "cores": out["cores"], "kind": "oracle",
                   "sample": cpu_sample_text(spec, args.cpu_window, out) + f" ({out['times'][0]:.1f} s measured)"}
            if args.workload in ("C1", "C2"):
                # the oracle's direct mode beside it: sparse LU of A once, then exact solves
                od = run_cpu_sample(args.workload, info["lambda_"], 1, args.cpu_window, nnz, solver="direct")
                cpu["direct"] = {"value": od["per_step_scaled"][0], "unit": UNIT, "cores": od["cores"],
                                 "factor_s_measured": round(od["factor_s"], 3),
                                 "sample": "the same windows, sparse-LU solves (A factored once before the step, "
                                           "not counted) instead of Jacobi-PCG, scaled the same way "
                                           f"({od['times'][0]:.2f} s measured)"}
        except Exception as ex:  # report, do not hide
            cpu = {"value": None, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": sec_per_outer, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(spec, world),
            "precision_path": "FP32 edge/SpMM/vectors, double-FP32 dots and PCG solution, FP64 P-step; "
                              + {"learned": "learned FSAI preconditioner (BF16 tensor-core MLP, weights "
                                            "paper_1612_06496_gb300/fsai_weights.npz)",
                                 "jacobi": "Jacobi preconditioner",
                                 "classical": "classical FSAI preconditioner",
                                 "ic0": "IC(0) preconditioner (level-scheduled triangular solves)"}[args.precond],
            "precond": args.precond,
            "pcg_iters_mean": iters_total / max(n_solves, 1),
            "pcg_iters_max": max(s["pcg_iters_max"] for s in stats),
            "pcg_relres_max": max(s["relres_max"] for s in stats),
            "pcg_replacements_per_solve": sum(s["replacements"] for s in stats) / max(n_solves, 1)
                                          * (len(stats[0].get("seg_iters", [])) or 1),
            "true_relres_fp64_max": true_relres,
            "gnnz_rhs_per_s": nnz_iters * d / (ms / 1e3) / 1e9,
            "setup_s": setup_s, "lambda": info["lambda_"], "r": info["r"],
            "fp32_other_precond": alt,
            "fp64": fp64,
            "speedup_vs_fp64": (fp64["sec_per_outer_iter"] / sec_per_outer) if fp64 else None,
            "roofline": roofline,
            "autotune": {k: {"spmm_variant": v[0], "spmm_ms": {str(a): round(b, 5) for a, b in v[1].items()},
                             "fsai_columns": {0: "slots", 1: "stencil"}[v[2]] if v[3] is not None and v[3][0] > 0
                             else None,
                             "fsai_ms": [round(float(x), 5) for x in v[3]] if v[3] is not None and v[3][0] > 0
                             else None,
                             "edge_columns": {0: "slots", 1: "stencil"}[v[4]],
                             # blocks per SM of each row kernel (0: its occupancy) and the times tried
                             "blocks_per_sm": {kk: {"chosen": b, "ms": {str(bb): round(t, 5) for bb, t in m.items()}}
                                               for kk, (b, m) in shapes.get(k, {}).items()},
                             "edge_ms": [round(float(x), 5) for x in v[5]] if v[5] is not None and v[5][0] > 0
                             else None}
                         for k, v in tuned.items()},
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
