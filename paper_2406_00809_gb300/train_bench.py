"""Training throughput on the 3-D anisotropic workload (64^3 = 262,144 unknowns,
-(u_xx + u_yy + 100 u_zz), 7-point stencil), and what the trained GNP buys.

    python -m paper_2406_00809_gb300.train_bench [--workload aniso64] [--steps 5000]

The GNP (8 Res-GCONV layers of width 16, MLPs of width 32) trains with the paper's
optimiser (Adam, lr 1e-3) on batches of 32 pairs (16 from Eq. 5 with 30 Arnoldi steps, 16
with x ~ N(0, I)).  Reported: milliseconds per training step (device-synchronised wall
time of gnp_train over all steps, after 3 warm-up steps), the best and the last-tenth
mean loss, and FGMRES(30) on b = A 1 to rtol 1e-8 with the trained GNP and with no
preconditioner (iterations, seconds).  One JSON line.  Inputs are synthetic
(paper_2406_00809_gb300.inputs).
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


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="aniso64")
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--maxiters", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=None, help="override the workload's batch")
    ap.add_argument("--arnoldi-m", type=int, default=None, help="override the workload's Arnoldi steps")
    args = ap.parse_args(argv)
    import torch
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp as g
    A, wl = I.workload(args.workload)
    Mt = g.mat_from_csr(A)
    cfg = g.make_config(L=wl.get("L", 8), batch=args.batch or wl.get("batch", 32),
                        arnoldi_m=args.arnoldi_m or wl.get("arnoldi_m", 30), lr=1e-3)
    M = g.gnp_create(Mt, cfg, I.init_weights(cfg.L, seed=0))
    g.gnp_train(M, 3)  # sampler set-up and first launches
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses, best = g.gnp_train_history(M, args.steps)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    g.gnp_train_release(M)
    b = torch.from_numpy(I.spmv(A, np.ones(A.n))).cuda()
    res = {}
    for name, P in (("gnp", M), ("none", None)):
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        g.fgmres_solve(Mt, b, x, P, restart=30, rtol=1e-8, maxiters=args.maxiters, history=False)  # capture
        x.zero_()
        info = g.fgmres_solve(Mt, b, x, P, restart=30, rtol=1e-8, maxiters=args.maxiters, history=False)
        res[name] = {"iters": info.iters, "status": info.status_name, "seconds": info.seconds,
                     "rel_res": info.rel_res_true}
    tail = max(1, len(losses) // 10)
    out = {"workload": args.workload, "n": A.n, "nnz": A.nnz, "batch": cfg.batch, "arnoldi_m": cfg.arnoldi_m,
           "steps": args.steps, "train_s": train_s, "ms_per_step": 1e3 * train_s / max(1, args.steps),
           "best_loss": best, "late_loss": float(np.mean(losses[-tail:])), "first_loss": float(losses[0]),
           "fgmres_gnp": res["gnp"], "fgmres_none": res["none"]}
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
