"""Pins of the Jacobi and inner-GMRES preconditioner oracle (Sec. 3 "Compared methods").

* Jacobi on a diagonal matrix is its exact inverse; a zero diagonal passes v through.
* Inner GMRES with as many steps as unknowns (and rtol = 0) solves A z = v exactly
  (dense solve); with fewer steps it equals the textbook GMRES(m) of the Krylov oracle
  (modified Gram-Schmidt, dense least squares) on one cycle; its residual is minimal
  over the Krylov space (random members of K_k do worse); the early stop takes the
  first k whose minimal residual meets rtol.
* FGMRES preconditioned by the exact inverse (inner GMRES with n steps) converges in one
  outer iteration; with Jacobi on a diagonal matrix likewise.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import krylov_ref as K
from oracle import precond_ref as P
from paper_2406_00809_gb300 import inputs as I


def test_jacobi_diagonal_inverse_and_zero_diagonal():
    d = np.array([2.0, -4.0, 0.0, 0.5])
    A = sp.csr_matrix(np.diag(d) + np.diag([1.0, 1.0, 1.0], 1))
    v = np.array([1.0, 2.0, 3.0, 4.0])
    z = P.jacobi(A)(v)
    np.testing.assert_array_equal(z, [0.5, -0.5, 3.0, 8.0])
    D = sp.diags([3.0, 5.0, 7.0]).tocsr()
    b = np.array([3.0, 10.0, 21.0])
    x, info = K.fgmres(D, b, P.jacobi(D), m=5, rtol=1e-12, maxiters=5)
    assert info["iters"] == 1 and info["status"] == K.OK
    np.testing.assert_allclose(x, [1.0, 2.0, 3.0], rtol=1e-15)


def test_inner_gmres_exact_with_n_steps():
    rng = np.random.default_rng(0)
    n = 8
    A = sp.csr_matrix(rng.normal(size=(n, n)) + 4 * np.eye(n))
    v = rng.normal(size=n)
    z, k, _ = P.inner_gmres_solve(A, v, iters=10, rtol=0.0)
    assert k <= n
    np.testing.assert_allclose(z, np.linalg.solve(A.toarray(), v), rtol=1e-10, atol=1e-12)
    # as a preconditioner it is the exact inverse: one outer iteration
    x, info = K.fgmres(A, v, P.inner_gmres(A, iters=10, rtol=0.0), m=5, rtol=1e-10, maxiters=5)
    assert info["iters"] == 1 and info["status"] == K.OK


def test_inner_gmres_equals_textbook_gmres_one_cycle():
    A = I.convdiff2d(12, 100.0).to_scipy()
    v = I.gaussian(A.shape[0], seed=4)
    for m in (1, 3, 10):
        z, k, _ = P.inner_gmres_solve(A, v, iters=m, rtol=0.0)
        x, hist = K.gmres_textbook(A, v, m=m, maxiters=m)
        assert k == m
        np.testing.assert_allclose(z, x, rtol=1e-9, atol=1e-12 * np.abs(x).max())


def test_inner_gmres_minimal_residual_and_first_k():
    A = I.poisson2d(10).to_scipy()
    v = I.gaussian(A.shape[0], seed=5)
    rtol = 1e-2
    z, k, res = P.inner_gmres_solve(A, v, iters=30, rtol=rtol)
    beta = np.linalg.norm(v)
    assert res <= rtol * beta
    assert np.linalg.norm(v - A @ z) == pytest.approx(res, rel=1e-8)
    # k is the first step count that meets rtol
    _, k1, res1 = P.inner_gmres_solve(A, v, iters=k - 1, rtol=0.0)
    assert k1 == k - 1 and res1 > rtol * beta
    # minimal over K_k: random members of span{v, Av, ...} (orthonormalised) do worse
    V, _ = K.arnoldi(A, v, k)
    rng = np.random.default_rng(1)
    for _ in range(20):
        c = rng.normal(size=k)
        zt = V[:, :k] @ c
        zt *= (zt @ (A.T @ v)) / np.linalg.norm(A @ zt) ** 2  # best multiple of zt
        assert np.linalg.norm(v - A @ zt) >= res * (1 - 1e-12)
    # zero vector
    z0, k0, r0 = P.inner_gmres_solve(A, np.zeros(A.shape[0]))
    assert k0 == 0 and r0 == 0.0 and not np.any(z0)
