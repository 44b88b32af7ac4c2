"""Training and evaluation of the learned FSAI preconditioner.

The network (4 -> 64 -> 64 -> 2, see include/pfe.h) is trained on the
system matrices the method itself builds: for each seeded synthetic image
the library builds the heat-kernel graph and A = lam M^T M + r D, then
returns the Kaporin criterion of G A G^T and its gradient (forward and
backward on the GPU, hidden layer on the tensor cores); the library's Adam
kernel updates the parameters.  Nothing here computes on the host beyond
bookkeeping: parameters, moments and gradients are device tensors.

    python -m paper_1612_06496_gb300.learned train --images 2000 --out fsai_weights.npz
    python -m paper_1612_06496_gb300.learned eval --weights fsai_weights.npz
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fsai_weights.npz")
SOFTPLUS_ONE = float(np.log(np.expm1(1.0)))


def init_params(seed: int = 0) -> np.ndarray:
    """He-initialised hidden layers, zero output layer and softplus(b3[1]) = 1:
    the untrained network is exactly the Jacobi preconditioner."""
    H = 64
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((4, H)) * np.sqrt(2.0 / 4)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    parts = [W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), np.zeros(2 * H), np.array([0.0, SOFTPLUS_ONE])]
    return np.concatenate(parts).astype(np.float32)


def training_specs(count: int, seed0: int = 40000):
    """Seeded training images of 128x128 to 481x321, radius 2 or 3."""
    from synth import ImageSpec
    out = []
    for k in range(count):
        seed = seed0 + k
        rng = np.random.default_rng(seed + 982451653)
        W = int(rng.integers(128, 482))
        H = int(rng.integers(128, 322))
        K = int(rng.integers(3, 13))
        radius = 3.0 if k % 2 == 0 else 2.0
        sigma = 0.08 if radius == 3.0 else 0.1
        out.append(ImageSpec(f"train{k}", H, W, K, 0.03, seed=seed, gradient=bool(k % 3 == 0),
                             texture=bool(k % 3 == 1), radius=radius, sigma=sigma, d=8))
    return out


def load_weights(path: str = WEIGHTS) -> np.ndarray:
    with np.load(path) as z:
        return z["params"].astype(np.float32)


def method_rhs(p, Y0, steps: int):
    """A right-hand side of Eq. 13 the method produces on this image: the
    next system's after `steps` inner iterations from Y0 (Jacobi PCG), as a
    device tensor (n x d FP64)."""
    import torch
    p.init(torch.from_numpy(Y0).cuda())
    for _ in range(steps):
        p.inner_step()
    return torch.from_numpy(np.ascontiguousarray(p.get("RHS"))).cuda()


def train(images: int, epochs: int, batch: int, lr: float, out: str, seed: int = 0, log=print,
          mu: float = 0.0, rhs_steps: int = 1, init: np.ndarray | None = None, first_image: int = 0) -> dict:
    import torch

    from paper_1612_06496_gb300 import PFE
    from paper_1612_06496_gb300.pfe import adam_update, fsai_param_count
    from synth import make_image, features_from_image, make_problem

    dev = torch.device("cuda")
    npar = fsai_param_count()
    params = torch.from_numpy(init_params(seed) if init is None else init.astype(np.float32)).to(dev)
    m = torch.zeros(npar, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    gsum = torch.zeros_like(m)
    gtmp = torch.zeros_like(m)
    specs = training_specs(first_image + images)[first_image:]
    step, hist = 0, []
    t0 = time.time()
    for ep in range(epochs):
        order = np.random.default_rng(seed + ep).permutation(len(specs))
        losses = []
        for bi in range(0, len(order), batch):
            gsum.zero_()
            nb = 0
            for k in order[bi:bi + batch]:
                s = specs[k]
                if mu > 0.0:  # Kaporin + mu x the residual on a right-hand side the method produced
                    X, Y0 = make_problem(s)
                    p = PFE(torch.from_numpy(X).to(dev), sigma=s.sigma, H=s.H, W=s.W, radius=s.radius,
                            precision="mixed")
                    B = method_rhs(p, Y0, rhs_steps)
                    loss, _, _ = p.fsai_loss_grad_rhs(params, B, mu, gtmp)
                else:
                    X = features_from_image(make_image(s))
                    p = PFE(torch.from_numpy(X).to(dev), sigma=s.sigma, H=s.H, W=s.W, radius=s.radius,
                            precision="mixed")
                    loss, _ = p.fsai_loss_grad(params, gtmp)
                p.close()
                gsum += gtmp
                losses.append(loss)
                nb += 1
            gsum /= nb
            step += 1
            adam_update(params, gsum, m, v, step, lr)
        torch.cuda.synchronize()
        hist.append({"epoch": ep, "mean_loss": float(np.mean(losses)), "seconds": time.time() - t0})
        log(json.dumps(hist[-1]))
    theta = params.cpu().numpy()
    meta = {"images": images, "first_image": first_image, "epochs": epochs, "batch": batch, "lr": lr, "seed": seed,
            "mu": mu, "rhs_steps": rhs_steps, "history": hist}
    if out:
        np.savez(out, params=theta, meta=json.dumps(meta))
    return {"params": theta, "meta": meta}


def evaluate(params: np.ndarray | None, specs, tol: float = 1e-6, n_inner: int = 10) -> list[dict]:
    """PCG iterations and solve time over the second outer iteration of each
    image (the first one runs untimed), for Jacobi (FP32), the learned FSAI
    (FP32), the untrained network (FP32; equals Jacobi), the classical FSAI
    on the same pattern (FP32) and plain FP64 Jacobi."""
    import torch

    from paper_1612_06496_gb300 import PFE
    from synth import make_problem

    dev = torch.device("cuda")
    rows = []
    for s in specs:
        X, Y0 = make_problem(s)
        Xd, Y0d = torch.from_numpy(X).to(dev), torch.from_numpy(Y0).to(dev)
        res = {"image": s.name, "n": s.n, "radius": s.radius, "d": s.d}
        arms = [("jacobi_fp32", "mixed", None), ("learned_fp32", "mixed", params),
                ("untrained_fp32", "mixed", init_params(0)), ("classical_fp32", "mixed", "classical"),
                ("jacobi_fp64", "fp64", None)]
        for name, prec, th in arms:
            if th is None and name == "learned_fp32":
                continue
            p = PFE(Xd, sigma=s.sigma, H=s.H, W=s.W, radius=s.radius, precision=prec, tol=tol)
            if isinstance(th, str):
                p.fsai_classical()
            elif th is not None:
                p.fsai_set(th)
            p.init(Y0d)
            p.solve(1, n_inner)  # first outer iteration (also builds the CUDA graph)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = p.solve(1, n_inner)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            res[name] = {"pcg_iters_mean": st["pcg_iters_total"] / max(st["n_solves"], 1),
                         "pcg_iters_max": st["pcg_iters_max"], "seconds": dt,
                         "converged": st["n_unconverged"] == 0}
            p.close()
        rows.append(res)
    return rows


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--images", type=int, default=2000)
    t.add_argument("--epochs", type=int, default=2)
    t.add_argument("--batch", type=int, default=8)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--out", default=WEIGHTS)
    e = sub.add_parser("eval")
    e.add_argument("--weights", default=WEIGHTS)
    e.add_argument("--images", type=int, default=10)
    a = ap.parse_args()
    if a.cmd == "train":
        train(a.images, a.epochs, a.batch, a.lr, a.out)
    else:
        from synth import CONFIGS
        from dataclasses import replace
        base = CONFIGS["C4"]
        specs = [replace(base, name=f"C4eval{k}", seed=49000 + k) for k in range(a.images)]
        print(json.dumps(evaluate(load_weights(a.weights), specs), indent=1))


if __name__ == "__main__":
    main()
