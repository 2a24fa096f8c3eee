"""The paper's solver-comparison protocol (Sec. 3) on the synthetic problem families.

    python -m paper_2406_00809_gb300.protocol [--problems poisson128,convdiff128,powerlaw32k,aniso24]
        [--train-steps 2000] [--restart 10] [--maxiters 100] [--rtol 1e-8] [--hprec fp32]

For each problem: the GNP is trained with the paper's hyperparameters (8 Res-GCONV
layers of width 16, MLPs of width 32, Adam 1e-3, batch 16 with 8 Arnoldi (m = 40) and 8
Gaussian pairs, `train-steps` steps, best-loss weights); its training time is the
construction time.  The test system has the solution x = 1 (b = A 1) and starts from
x0 = 0.  Four right preconditioners run through the same FGMRES(restart): none, Jacobi,
inner GMRES (10 steps, 1e-6) and the GNP.

* Run 1 stops at rtol or maxiters (100) and reports Iter-AUC.
* Run 2 disables maxiters and stops at rtol or a time limit equal to the longest
  run-1 solve among the four preconditioners, and reports Time-AUC.

Times are the device clock of the solve (per-iteration timestamps taken by the kernel
that ends each iteration); every configuration runs once untimed first so that CUDA-graph
capture is not counted.  One JSON line per (problem, preconditioner), then one summary
line per problem naming the best preconditioner by each metric.  Inputs are synthetic
(paper_2406_00809_gb300.inputs); the paper's SuiteSparse matrices are not used.
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
    "poisson128": lambda: I.poisson2d(128),
    "convdiff128": lambda: I.convdiff2d(128, 100.0),
    "powerlaw32k": lambda: I.powerlaw(32768, seed=11),
    "aniso24": lambda: I.aniso3d(24, 100.0),
    "poisson32": lambda: I.poisson2d(32),
    "convdiff32": lambda: I.convdiff2d(32, 100.0),
}
PRECONDS = ("none", "jacobi", "gmres", "gnp")


def run_problem(g, name, A, args):
    import torch
    Mt = g.mat_from_csr(A)
    cfg = g.make_config(L=8, batch=16, arnoldi_m=40, lr=1e-3, seed=args.seed)
    M = g.gnp_create(Mt, cfg, I.init_weights(8, seed=args.seed))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best = g.gnp_train(M, args.train_steps) if args.train_steps > 0 else float("nan")
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    g.gnp_train_release(M)
    g.gnp_set_hprec(M, g.H_BF16 if args.hprec == "bf16" else g.H_FP32)
    P = {"none": None,
         "jacobi": g.gnp_precond_create(Mt, g.PRECOND_JACOBI),
         "gmres": g.gnp_precond_create(Mt, g.PRECOND_GMRES, inner_iters=10, inner_rtol=1e-6),
         "gnp": g.gnp_precond_create(Mt, g.PRECOND_GNP, M=M)}
    b = torch.from_numpy(I.spmv(A, np.ones(A.n))).cuda()
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    ones = torch.ones(A.n, dtype=torch.float64, device="cuda")

    def solve(p, maxiters, timeout):
        x.zero_()
        g.fgmres_solve(Mt, b, x, P[p], restart=args.restart, rtol=args.rtol, maxiters=maxiters,
                       timeout=timeout, times=True)  # untimed: graph capture
        x.zero_()
        info = g.fgmres_solve(Mt, b, x, P[p], restart=args.restart, rtol=args.rtol, maxiters=maxiters,
                              timeout=timeout, times=True)
        err = float((x - ones).norm() / ones.norm())
        return info, err

    run1 = {}
    for p in PRECONDS:
        info, err = solve(p, args.maxiters, 0.0)
        run1[p] = dict(iters=info.iters, status=info.status_name, rel_res=info.rel_res_true, x_err=err,
                       iter_auc=g.iter_auc(info.history, args.rtol), time_s=float(info.times[-1]))
    limit = max(r["time_s"] for r in run1.values())
    run2 = {}
    for p in PRECONDS:
        info, err = solve(p, args.cap, limit)
        run2[p] = dict(iters=info.iters, status=info.status_name, rel_res=info.rel_res_true, x_err=err,
                       time_auc=g.time_auc(info.history, info.times, args.rtol), time_s=float(info.times[-1]))
    for p in PRECONDS:
        print(json.dumps({"problem": name, "n": A.n, "nnz": A.nnz, "precond": p,
                          "maxiters_run": run1[p], "timeout_run": run2[p],
                          "construction_s": train_s if p == "gnp" else None,
                          "best_train_loss": best if p == "gnp" else None}), flush=True)
    print(json.dumps({"problem": name, "timeout_s": limit, "train_steps": args.train_steps,
                      "best_by_iter_auc": min(PRECONDS, key=lambda p: run1[p]["iter_auc"]),
                      "best_by_time_auc": min(PRECONDS, key=lambda p: run2[p]["time_auc"])}), flush=True)
    return run1, run2


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", default="poisson128,convdiff128,powerlaw32k,aniso24")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--restart", type=int, default=10)
    ap.add_argument("--maxiters", type=int, default=100)
    ap.add_argument("--cap", type=int, default=100000, help="iteration bound of the time-limited run")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--hprec", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp as g
    out = {}
    for name in args.problems.split(","):
        out[name] = run_problem(g, name, PROBLEMS[name](), args)
    return out


if __name__ == "__main__":
    main()
