"""Throughput of multi-right-hand-side FGMRES: k systems with one matrix and one GNP.

    python -m paper_2406_00809_gb300.multi_bench [--workload convdiff256] [--ks 1,2,4,8]
        [--train-steps 2000] [--reps 3]

The GNP is trained as in the solve benchmark (Sec. 3 hyperparameters); then for each k the
k right-hand sides b_r = A x_r (x_r ~ N(0, I), seeds 0..k-1) are solved to rtol 1e-8 by
FGMRES(30): k = 1 through fgmres_solve, k > 1 through fgmres_solve_multi.  Inputs are
resident on the device; the L2 cache is flushed (256 MB write) before every timed call.
Reported per k: the median wall time of a call (CUDA events), solves per second, the
speed-up in solves per second over k = 1, and the iteration counts.  One JSON line per k.
Inputs are synthetic (paper_2406_00809_gb300.inputs).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2406_00809_gb300 import inputs as I  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="convdiff256")
    ap.add_argument("--ks", default="1,2,4,8")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--maxiters", type=int, default=3000)
    ap.add_argument("--identity", action="store_true", help="no preconditioner")
    args = ap.parse_args(argv)
    import torch
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp as g
    A, _ = I.workload(args.workload)
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = []
    with torch.cuda.stream(stream):
        Mt = g.mat_from_csr(A)
        M = None
        if not args.identity:
            M = g.gnp_create(Mt, g.make_config(L=8, batch=16, arnoldi_m=40), I.init_weights(8, seed=0))
            g.gnp_train(M, args.train_steps)
            g.gnp_train_release(M)
        kmax = max(int(k) for k in args.ks.split(","))
        xs = np.stack([I.gaussian(A.n, seed=r) for r in range(kmax)], axis=1)
        Ball = np.stack([I.spmv(A, xs[:, r]) for r in range(kmax)], axis=1)
        base = None
        for k in (int(v) for v in args.ks.split(",")):
            B = torch.from_numpy(np.ascontiguousarray(Ball[:, :k])).cuda()
            X = torch.zeros_like(B)
            b1 = B[:, 0].contiguous()
            x1 = torch.zeros_like(b1)
            times, iters, stats = [], None, None
            for rep in range(args.reps + 1):
                X.zero_()
                x1.zero_()
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if k == 1:
                    info = g.fgmres_solve(Mt, b1, x1, M, restart=args.restart,
                                          rtol=1e-8, maxiters=args.maxiters, stream=stream, history=False)
                    infos = [info]
                else:
                    infos = g.fgmres_solve_multi(Mt, B, X, M, restart=args.restart, rtol=1e-8,
                                                 maxiters=args.maxiters, stream=stream, history=False)
                e1.record(stream)
                e1.synchronize()
                if rep > 0:  # the first call captures the graphs
                    times.append(e0.elapsed_time(e1) / 1e3)
                iters = [i.iters for i in infos]
                stats = [i.status_name for i in infos]
            t = statistics.median(times)
            sps = k / t
            if base is None:
                base = sps
            row = {"workload": args.workload, "n": A.n, "k": k, "preconditioner": "none" if M is None else "gnp",
                   "seconds_per_call": t, "solves_per_s": sps, "speedup_vs_k1": sps / base, "iters": iters,
                   "status": stats}
            out.append(row)
            print(json.dumps(row), flush=True)
    return out


if __name__ == "__main__":
    main()
