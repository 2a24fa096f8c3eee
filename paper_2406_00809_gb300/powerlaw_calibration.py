"""Calibrate the diagonal shift of the power-law workload so that cond(A) ~ 1e6.

The general sparse workload is A = P (E + D + s I) P^T with power-law row lengths,
N(0, 1) off-diagonal values E and an N(0, 1) diagonal D (``inputs.powerlaw``).  The
shift is stated as a fraction f of the circular-law radius rho = sqrt(sum a_ij^2 / n)
of the unshifted matrix, s = f * rho, so that one number serves every size.

For n = 4,096 and 16,384 (seed 0) this script finds s with cond_2(A) = 1e6 by bisection
on s in [0, rho] (cond falls as the shift moves the spectrum off the origin):
* sigma_max from ARPACK on the sparse A (``svds``);
* sigma_min from the dense LU of A and Lanczos on (A^T A)^{-1} (``eigsh``), which gives
  the same smallest singular value as a full dense SVD at a fraction of its cost.
The calibrated fraction at each size is s / rho; the stored fraction is their geometric
mean.  At each calibrated shift a full dense SVD (``scipy.linalg.svdvals``) confirms the
condition number.  At n = 2^20 the script records rho, s and sigma_max; sigma_min, and so
cond, are not computed there (the dense or factored forms do not fit), and the record
says so.

The permutation does not change singular values, so the calibration runs on the
unpermuted matrix.  Problem set-up only: nothing here is the method's arithmetic.

Run: python -m paper_2406_00809_gb300.powerlaw_calibration [--no-full-svd]
Writes paper_2406_00809_gb300/powerlaw_shift.json.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import scipy.linalg as sl
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from . import inputs as I

TARGET_COND = 1e6
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "powerlaw_shift.json")


def unshifted(n: int, seed: int = 0):
    rows, cols, vals, diag, _ = I.powerlaw_unshifted(n, seed=seed)
    E = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return E, diag, I.powerlaw_radius(vals, diag)


def sigma_max(A: sp.csr_matrix) -> float:
    return float(sla.svds(A, k=1, which="LM", return_singular_vectors=False, tol=1e-10)[0])


def sigma_min(A: sp.csr_matrix) -> float:
    n = A.shape[0]
    lu = sl.lu_factor(A.toarray(), check_finite=False)

    def inv_ata(x):
        y = sl.lu_solve(lu, x, trans=1, check_finite=False)   # A^{-T} x
        return sl.lu_solve(lu, y, trans=0, check_finite=False)  # A^{-1} A^{-T} x

    op = sla.LinearOperator((n, n), matvec=inv_ata, dtype=np.float64)
    lam = sla.eigsh(op, k=1, which="LM", return_eigenvectors=False, tol=1e-10)[0]
    return float(1.0 / np.sqrt(lam))


def cond_at(E, diag, s):
    n = diag.size
    A = (E + sp.diags(diag + s)).tocsr()
    return sigma_max(A), sigma_min(A)


def calibrate(n: int, steps: int = 14, full_svd: bool = True) -> dict:
    E, diag, rho = unshifted(n)
    lo, hi = 0.0, rho
    smx, smn = cond_at(E, diag, lo)
    k_lo = smx / smn
    smx, smn = cond_at(E, diag, hi)
    k_hi = smx / smn
    if not (k_lo > TARGET_COND > k_hi):
        raise RuntimeError(f"n={n}: cond(0)={k_lo:.3e}, cond(rho)={k_hi:.3e} do not bracket {TARGET_COND:g}")
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        smx, smn = cond_at(E, diag, mid)
        if smx / smn > TARGET_COND:
            lo = mid
        else:
            hi = mid
        print(f"  n={n} s={mid:.6f} cond={smx / smn:.3e}", flush=True)
    s = 0.5 * (lo + hi)
    smx, smn = cond_at(E, diag, s)
    rec = dict(n=n, rho=rho, shift=s, fraction=s / rho, sigma_max=smx, sigma_min=smn, cond=smx / smn,
               cond_at_zero_shift=k_lo)
    if full_svd:
        t = time.time()
        sv = sl.svdvals((E + sp.diags(diag + s)).toarray(), check_finite=False)
        rec["cond_dense_svd"] = float(sv[0] / sv[-1])
        rec["dense_svd_seconds"] = time.time() - t
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--no-full-svd", action="store_true")
    ap.add_argument("--sizes", default="4096,16384")
    args = ap.parse_args()
    recs = []
    for n in [int(t) for t in args.sizes.split(",")]:
        t = time.time()
        r = calibrate(n, full_svd=not args.no_full_svd)
        r["seconds"] = time.time() - t
        print(json.dumps(r), flush=True)
        recs.append(r)
    frac = float(np.exp(np.mean([np.log(r["fraction"]) for r in recs])))
    E, diag, rho = unshifted(1 << 20)
    s = frac * rho
    A = (E + sp.diags(diag + s)).tocsr()
    big = dict(n=1 << 20, rho=rho, shift=s, sigma_max=sigma_max(A),
               note="sigma_min and cond not computed at this size (no dense or factored form fits); "
                    "cond is estimated, not verified")
    out = dict(fraction=frac, target_cond=TARGET_COND, calibration=recs, full_size=big,
               method="bisection on s: sigma_max by ARPACK svds, sigma_min by dense LU + Lanczos on "
                      "(A^T A)^-1; confirmed by a full dense SVD at the calibrated shift")
    json.dump(out, open(OUT, "w"), indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
