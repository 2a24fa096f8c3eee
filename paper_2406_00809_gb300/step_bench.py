"""Cost of one GNP-preconditioned FGMRES step (Algorithm 1) on a workload.

    python -m paper_2406_00809_gb300.step_bench [--workload convdiff256] [--iters 60]
        [--restart 30] [--reps 4] [--hprec fp32|bf16]

Runs `reps` solves of exactly `iters` Arnoldi steps (rtol = 0, so no early exit) with a
randomly initialised GNP (Sec. 2.3: the per-step cost depends on the matrix, L, the
restart length and the hidden-block precision, not on the trained weights) and prints
one JSON line per solve with the CUDA-event time per step.  The launch sequence is fixed
(per solve: 2 + cycles * (restart * (L + 3) + 3) kernels), which makes it the command to
put under ncu for a per-kernel breakdown of a step.  Inputs are synthetic
(paper_2406_00809_gb300.inputs).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2406_00809_gb300 import inputs as I  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="convdiff256")
    ap.add_argument("--iters", type=int, default=60)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--reps", type=int, default=4)
    ap.add_argument("--L", type=int, default=8)
    ap.add_argument("--hprec", default="fp32", choices=["fp32", "bf16"])
    a = ap.parse_args()
    import torch
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp
    A, _ = I.workload(a.workload)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=a.L), I.init_weights(a.L, seed=0))
    gnp.gnp_set_hprec(M, gnp.H_BF16 if a.hprec == "bf16" else gnp.H_FP32)
    b = torch.from_numpy(I.spmv(A, I.gaussian(A.n, seed=0))).cuda()
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    for rep in range(a.reps):
        x.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        info = gnp.fgmres_solve(Mt, b, x, M, restart=a.restart, rtol=0.0, maxiters=a.iters, history=False)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        print(json.dumps({"workload": a.workload, "n": A.n, "nnz": A.nnz, "L": a.L, "hprec": a.hprec,
                          "restart": a.restart, "rep": rep, "iters": info.iters, "cycles": info.cycles,
                          "ms": ms, "us_per_step": 1000.0 * ms / max(1, info.iters)}), flush=True)


if __name__ == "__main__":
    main()
