"""GNP-FGMRES on the 2^20-row power-law workload: does it reach rtol 1e-8?

    python -m paper_2406_00809_gb300.powerlaw_study [--train-steps 2000] [--maxiters 3000]

The matrix is inputs.powerlaw(2^20): N(0, 1) values, power-law row lengths (mean 12,
max 2,000) and the diagonal shift that gives cond_2 ~ 1e6 at the calibration sizes.
This script solves b = A x (x ~ N(0, 1), seed 0) with FGMRES(50) to rtol 1e-8
(Algorithm 1) three ways -- no preconditioner, and the GNP (8 layers, hidden width 16)
trained by this library for --train-steps Adam steps (batch 16, half Eq. 5 samples with
m = 40, half N(0, I); Sec. 3) with a float32 and with a bfloat16 hidden block -- and
prints one JSON line per solve: status, iterations, seconds, the true relative residual
and the relative residual every 100 iterations.  It also reports where the spectrum of a
smaller matrix of the same construction lies (eigenvalues of the n = 4,096 instance).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs as I


def spectrum_note(n: int = 4096) -> dict:
    A = I.powerlaw(n, seed=0).to_scipy().toarray()
    ev = np.linalg.eigvals(A)
    return {"n": n, "min_real": float(ev.real.min()), "max_real": float(ev.real.max()),
            "max_abs_imag": float(np.abs(ev.imag).max()),
            "eigenvalues_left_of_origin": int((ev.real < 0).sum()),
            "eigenvalues_right_of_origin": int((ev.real > 0).sum())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--maxiters", type=int, default=3000)
    ap.add_argument("--log2n", type=int, default=20)
    a = ap.parse_args()
    import torch
    from . import build
    build.build()
    from . import gnp
    print(json.dumps({"spectrum_of_smaller_instance": spectrum_note()}), flush=True)
    t = time.perf_counter()
    A = I.powerlaw(1 << a.log2n, seed=0)
    b_np = I.spmv(A, I.gaussian(A.n, seed=0))
    print(json.dumps({"n": A.n, "nnz": A.nnz, "generate_s": time.perf_counter() - t}), flush=True)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=8, batch=16, arnoldi_m=40, seed=0), I.init_weights(8, seed=0))
    b = torch.from_numpy(b_np).cuda()
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    As = A.to_scipy()

    def solve(prec, label):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = gnp.fgmres_solve(Mt, b, x, prec, restart=50, rtol=1e-8, maxiters=a.maxiters)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        h = np.asarray(info.history)
        rr = float(np.linalg.norm(b_np - As @ x.cpu().numpy()) / np.linalg.norm(b_np))
        print(json.dumps({"solve": label, "status": info.status_name, "iters": info.iters, "seconds": dt,
                          "rel_res_true": rr,
                          "history_every_100": {int(i): float(h[i]) for i in
                                                list(range(0, len(h), 100)) + [len(h) - 1]}}), flush=True)

    solve(None, "M = I")
    t = time.perf_counter()
    losses, best = gnp.gnp_train_history(M, a.train_steps)
    torch.cuda.synchronize()
    print(json.dumps({"train_steps": a.train_steps, "train_s": time.perf_counter() - t, "best_loss": best,
                      "loss_every_10pct": [float(losses[i]) for i in
                                           range(0, len(losses), max(1, len(losses) // 10))]}), flush=True)
    solve(M, "GNP float32 hidden block")
    gnp.gnp_set_hprec(M, gnp.H_BF16)
    solve(M, "GNP bfloat16 hidden block")


if __name__ == "__main__":
    main()
