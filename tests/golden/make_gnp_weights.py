"""Write tests/golden/gnp_convdiff64_weights.npy: GNP weights trained by the oracle alone.

The GPU parity tests of preconditioned FGMRES need trained weights that do not come from
the CUDA path.  This script trains the paper's GNP (L = 8 Res-GCONV layers of Eq. 7,
hidden width 16, Sec. 3 "Hyperparameters") with the float64 oracle only: Adam with
lr 1e-3 for 2,000 steps, batch 16 = 8 pairs from Eq. 5 (Arnoldi with m = 40, reading
c11) and 8 pairs with x ~ N(0, I) (Sec. 3), the l1 residual loss, and the weights of the
lowest-loss step kept (reading c14).  Training system: 2-D convection-diffusion on a
64 x 64 grid (upwind, beta = 100), A_hat = A / gamma (Eq. 6).  Seeds: initial weights 0,
Philox sampler seed 0.

Run: python tests/golden/make_gnp_weights.py   (about 20-30 minutes on 8 cores)
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import gnp_ref as G  # noqa: E402
from oracle import krylov_ref as K  # noqa: E402
from paper_2406_00809_gb300 import inputs as I  # noqa: E402

L, STEPS, M_ARNOLDI, HALF = 8, 2000, 40, 8
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gnp_convdiff64_weights.npy")


def main():
    A = I.convdiff2d(64, 100.0)
    Ah = G.normalise(A.to_scipy())
    V, Hb = K.arnoldi(Ah, K.arnoldi_v1(A.n, 0), M_ARNOLDI)
    Q, _ = K.sampler_matrix(Hb)
    w = I.init_weights(L, seed=0).astype(np.float64)
    opt = G.Adam(w.size)
    best_loss, best_w = np.inf, w.copy()
    for step in range(STEPS):
        x = K.training_x(V, Q, HALF, HALF, 0, step)
        w_next, loss = G.train_step(Ah, w, L, G.FORM_PAPER, x, opt)
        if loss < best_loss:
            best_loss, best_w = loss, w.copy()
        w = w_next
        if step % 100 == 0:
            print(f"step {step} loss {loss:.5f} best {best_loss:.5f}", flush=True)
    np.save(OUT, best_w.astype(np.float32))
    print(f"best loss {best_loss:.6f} -> {OUT}")


if __name__ == "__main__":
    main()
