"""The ablations of Sec. 4 ("Are the proposed training-data generation and the
scale-equivariance design necessary?", Fig. 6) on the synthetic problem families.

    python -m paper_2406_00809_gb300.ablation [--problems poisson64,convdiff64,aniso16,powerlaw8k]
        [--train-steps 1000] [--restart 10] [--maxiters 100] [--rtol 1e-8]

Variants (gnp_config.sample_mode / no_scale):
* mix       the paper's method: B/2 Eq. 5 pairs and B/2 pairs with x ~ N(0, I), with s;
* x_normal  all B pairs with x ~ N(0, I), with s;
* b_normal  all B right-hand sides b ~ N(0, I), with s;
* no_scale  the paper's sampling without the scaling s of Eq. 8.

For every problem and variant: the training loss (best, and the mean over the last tenth
of the steps) and the preconditioner's quality on the paper's test system (x = 1,
x0 = 0, FGMRES(restart), rtol, maxiters): final relative residual, iterations and
Iter-AUC.  Every variant starts from the same initial weights and uses the same seed.
One JSON line per (problem, variant), then a line with each variant's median over the
problems.  Inputs are synthetic (paper_2406_00809_gb300.inputs).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2406_00809_gb300 import inputs as I  # noqa: E402

PROBLEMS = {
    "poisson64": lambda: I.poisson2d(64),
    "convdiff64": lambda: I.convdiff2d(64, 100.0),
    "aniso16": lambda: I.aniso3d(16, 100.0),
    "powerlaw8k": lambda: I.powerlaw(8192, seed=21),
    "poisson16": lambda: I.poisson2d(16),
}
VARIANTS = {"mix": (0, False), "x_normal": (1, False), "b_normal": (2, False), "no_scale": (0, True)}


def run(g, name, A, variant, args):
    import torch
    mode, no_scale = VARIANTS[variant]
    Mt = g.mat_from_csr(A)
    cfg = g.make_config(L=8, batch=16, arnoldi_m=40, lr=1e-3, seed=args.seed, sample_mode=mode,
                        no_scale=no_scale)
    M = g.gnp_create(Mt, cfg, I.init_weights(8, seed=args.seed))
    t0 = time.perf_counter()
    losses, best = g.gnp_train_history(M, args.train_steps)
    train_s = time.perf_counter() - t0
    g.gnp_train_release(M)
    b = torch.from_numpy(I.spmv(A, np.ones(A.n))).cuda()
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = g.fgmres_solve(Mt, b, x, M, restart=args.restart, rtol=args.rtol, maxiters=args.maxiters)
    tail = max(1, len(losses) // 10)
    return {"problem": name, "n": A.n, "variant": variant, "sample_mode": mode, "no_scale": no_scale,
            "train_steps": args.train_steps, "train_s": train_s, "best_loss": best,
            "late_loss": float(np.mean(losses[-tail:])) if len(losses) else None,
            "rel_res": info.rel_res_true, "iters": info.iters, "status": info.status_name,
            "iter_auc": g.iter_auc(info.history, args.rtol)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", default="poisson64,convdiff64,aniso16,powerlaw8k")
    ap.add_argument("--variants", default=",".join(VARIANTS))
    ap.add_argument("--train-steps", type=int, default=1000)
    ap.add_argument("--restart", type=int, default=10)
    ap.add_argument("--maxiters", type=int, default=100)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp as g
    rows = []
    for name in args.problems.split(","):
        A = PROBLEMS[name]()
        for v in args.variants.split(","):
            r = run(g, name, A, v, args)
            rows.append(r)
            print(json.dumps(r), flush=True)
    summary = {}
    for v in args.variants.split(","):
        rs = [r for r in rows if r["variant"] == v]
        summary[v] = {k: float(np.median([r[k] for r in rs])) for k in ("best_loss", "late_loss", "rel_res",
                                                                        "iter_auc")}
    print(json.dumps({"summary_median_over_problems": summary}), flush=True)
    return rows


if __name__ == "__main__":
    main()
