"""Write tests/golden/gnp_iteration_bands.json: iteration counts of the float64 oracle's
GNP-preconditioned FGMRES (Algorithm 1) with the oracle-trained weights of
gnp_convdiff64_weights.npy, and how far float32-level changes of the preconditioner
output move them.

Why a band: with a trained GNP the count of a restarted FGMRES run to rtol 1e-8 depends
on rounding at the level of float32.  On the 256 x 256 convection-diffusion system the
oracle's own count moves by tens of iterations when its z = M(v) is rounded to float32
or multiplied by (1 + 1e-7 xi), xi ~ N(0, 1) -- perturbations of the size of the float32
arithmetic that the GPU's GNP runs in.  Each record lists the counts of:
  f64        the oracle as it stands;
  z_f32      z rounded to float32 (the GPU stores the FGMRES directions Z in float32);
  noise<s>   z * (1 + 1e-7 xi), numpy seed s;
and for the bfloat16 hidden block the same with hstore='bf16' (reading c18: every stored
hidden block rounded to bfloat16, nearest even).  The GPU tests require the GPU's count
within [min - 2, max + 2] of its record.

Records:
  convdiff256_fp32 / convdiff256_bf16: 2-D convection-diffusion 256 x 256 (beta = 100),
      b = A x with x ~ N(0, 1) seed 0, FGMRES(30), rtol 1e-8, at most 3000 iterations;
  convdiff64_rhs<r>: the 64 x 64 problem, right-hand side r of inputs.rhs_set(A, 8, 20),
      FGMRES(20), rtol 1e-8, at most 1500 iterations (float32 hidden block).

Run: python tests/golden/make_iteration_bands.py [--jobs 4]   (oracle only; ~30 min)
"""
import argparse
import json
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

WEIGHTS = os.path.join(HERE, "gnp_convdiff64_weights.npy")
OUT = os.path.join(HERE, "gnp_iteration_bands.json")
L = 8


def _solve(task):
    from oracle import gnp_ref as G
    from oracle import krylov_ref as K
    from paper_2406_00809_gb300 import inputs as I
    record, variant, nx, rhs, m, maxit = task
    A = I.convdiff2d(nx, 100.0)
    b = I.spmv(A, I.gaussian(A.n, seed=0)) if rhs < 0 else I.rhs_set(A, 8, 20)[:, rhs]
    Ah = G.normalise(A.to_scipy())
    P = G.unpack(np.load(WEIGHTS), L)
    hstore = "bf16" if record.endswith("bf16") else "f64"
    M64 = lambda v: G.forward(Ah, v, P, G.FORM_PAPER, hstore=hstore)  # noqa: E731
    if variant == "f64":
        M = M64
    elif variant == "z_f32":
        M = lambda v: M64(v).astype(np.float32).astype(np.float64)  # noqa: E731
    else:
        rng = np.random.default_rng(int(variant[5:]))
        M = lambda v: (lambda z: z * (1.0 + 1e-7 * rng.standard_normal(z.size)))(M64(v))  # noqa: E731
    _, info = K.fgmres(A.to_scipy(), b, M, m=m, rtol=1e-8, maxiters=maxit)
    return record, variant, int(info["iters"]), int(info["status"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=4)
    a = ap.parse_args()
    variants = ["f64", "z_f32", "noise1", "noise2", "noise3"]
    tasks = [(f"convdiff256_{p}", v, 256, -1, 30, 3000) for p in ("fp32", "bf16") for v in variants]
    tasks += [(f"convdiff64_rhs{r}", v, 64, r, 20, 1500) for r in range(8) for v in variants]
    out = {}
    with ProcessPoolExecutor(max_workers=a.jobs) as ex:
        for record, variant, iters, status in ex.map(_solve, tasks):
            out.setdefault(record, {})[variant] = {"iters": iters, "status": status}
            print(record, variant, iters, status, flush=True)
    json.dump(out, open(OUT, "w"), indent=1, sort_keys=True)
    print("->", OUT)


if __name__ == "__main__":
    main()
