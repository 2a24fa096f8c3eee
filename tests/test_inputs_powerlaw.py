"""The general sparse workload generator (inputs.powerlaw) against its stated construction.

* row lengths (diagonal included) in [2, 2000] with mean 12 (the fitted power law);
* every row holds its diagonal and distinct columns; the matrix is square CSR;
* the values are N(0, 1) except the diagonal, which is N(0, 1) plus the shift
  s = fraction * rho, rho the circular-law radius of the unshifted matrix;
* P A P^T: a symmetric permutation keeps the shift on the diagonal and the singular
  values unchanged;
* the stored calibration reproduces cond_2(A) ~ 1e6 at n = 4,096 (sigma_min from a dense
  LU, independent of the calibration's bisection).
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl

from paper_2406_00809_gb300 import inputs as I

SHIFT_JSON = os.path.join(os.path.dirname(I.__file__), "powerlaw_shift.json")


def test_row_lengths_and_structure():
    A = I.powerlaw(1 << 16, seed=0)
    lens = np.diff(A.row_ptr)
    assert lens.min() >= 2 and lens.max() <= 2000
    assert abs(lens.mean() - 12.0) < 0.3, lens.mean()
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.col.size == A.val.size
    for i in range(0, A.n, 997):
        cols = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert i in cols                       # the diagonal (the shift lives there)
        assert np.all(np.diff(cols) > 0)       # sorted, distinct


def test_values_and_shift():
    n = 1 << 15
    rows, cols, vals, diag, _ = I.powerlaw_unshifted(n, seed=3)
    frac = json.load(open(SHIFT_JSON))["fraction"]
    s = frac * I.powerlaw_radius(vals, diag)
    A = I.powerlaw(n, seed=3, permute=False).to_scipy()
    d = A.diagonal()
    np.testing.assert_allclose(d - diag, s, rtol=0, atol=1e-12)
    off = A - __import__("scipy.sparse", fromlist=["diags"]).diags(d)
    v = off.data[off.data != 0]
    assert abs(v.mean()) < 0.01 and abs(v.std() - 1.0) < 0.01      # N(0, 1)
    assert abs(diag.mean()) < 0.05 and abs(diag.std() - 1.0) < 0.05
    # rho^2 = mean squared row norm: equals (nnz_off + n) / n for unit-variance values
    assert abs(I.powerlaw_radius(vals, diag) ** 2 - (vals.size + n) / n) < 0.05 * (vals.size + n) / n


def test_permutation_is_symmetric():
    A = I.powerlaw(4096, seed=5).to_scipy().toarray()
    B = I.powerlaw(4096, seed=5, permute=False).to_scipy().toarray()
    assert sorted(np.diag(A)) == sorted(np.diag(B))      # P A P^T keeps the diagonal
    np.testing.assert_allclose(sl.svdvals(A)[[0, -1]], sl.svdvals(B)[[0, -1]], rtol=1e-9)


@pytest.mark.parametrize("n", [4096])
def test_calibrated_condition_number(n):
    rec = {r["n"]: r for r in json.load(open(SHIFT_JSON))["calibration"]}[n]
    rows, cols, vals, diag, _ = I.powerlaw_unshifted(n, seed=0)
    A = np.zeros((n, n))
    A[rows, cols] = vals
    A[np.arange(n), np.arange(n)] = diag + rec["shift"]
    # sigma_max by power iteration on A^T A, sigma_min by inverse iteration on it (dense LU)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(n)
    for _ in range(300):
        x = A.T @ (A @ x)
        x /= np.linalg.norm(x)
    smax = np.linalg.norm(A @ x)
    lu = sl.lu_factor(A)
    y = rng.standard_normal(n)
    for _ in range(60):
        y = sl.lu_solve(lu, sl.lu_solve(lu, y, trans=1))
        y /= np.linalg.norm(y)
    smin = np.linalg.norm(A @ y)  # y: the right singular vector of sigma_min
    cond = smax / smin
    assert abs(cond / rec["cond_dense_svd"] - 1.0) < 1e-3, (cond, rec["cond_dense_svd"])
    assert 5e5 < cond < 2e6
