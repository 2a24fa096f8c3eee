"""Pins for the FGMRES / Arnoldi / sampler oracle (oracle/krylov_ref.py).

Expected values come from the mathematics of Sec. 2.1-2.2 (Eq. 1, Eq. 4, Eq. 5, the
proof of Theorem 1), from a separately written textbook GMRES that uses a dense
least-squares routine instead of Givens rotations, or from dense linear algebra.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gnp_ref as G
from oracle import krylov_ref as K
from oracle import philox_ref as PH
from paper_2406_00809_gb300 import inputs as I


def _gnp_op(A, L=2, seed=0, form=0):
    Ahat = G.normalise(A)
    P = G.unpack(I.init_weights(L, seed=seed), L)
    return lambda v: G.forward(Ahat, v, P, form)


def test_identity_preconditioner_is_gmres_iterate_for_iterate():
    # Eq. 1 with M = I reduces to Eq. 4: FGMRES must reproduce textbook GMRES
    A = I.convdiff2d(8, 100.0).to_scipy()
    b = np.random.default_rng(0).standard_normal(A.shape[0])
    _, hist = K.gmres_textbook(A, b, m=10, maxiters=30)
    for orth in ("mgs", "cgs2"):
        _, info = K.fgmres(A, b, None, m=10, rtol=1e-30, maxiters=30, orth=orth)
        h = np.array(info["history"])
        assert len(h) == 31
        np.testing.assert_allclose(h, hist, rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("orth", ["mgs", "cgs2"])
def test_arnoldi_relation_and_orthonormality(orth):
    A = I.convdiff2d(8, 100.0).to_scipy()
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    M = _gnp_op(A)
    _, info = K.fgmres(A, b, M, m=12, rtol=1e-30, maxiters=36, orth=orth, record=True)
    assert len(info["cycles"]) == 3
    for c in info["cycles"]:
        V, Z, Hb = c["V"], c["Z"], c["Hbar"]
        AZ = A @ Z
        assert np.linalg.norm(AZ - V @ Hb) <= 1e-12 * np.linalg.norm(AZ)
        assert np.abs(V.T @ V - np.eye(V.shape[1])).max() <= 1e-12
        # upper Hessenberg
        assert np.all(np.tril(Hb, -2) == 0)


def test_residual_nonincreasing_within_cycle_and_matches_true():
    A = I.convdiff2d(10, 100.0).to_scipy()
    b = np.random.default_rng(2).standard_normal(A.shape[0])
    M = _gnp_op(A, L=3, seed=2)
    m = 10
    x, info = K.fgmres(A, b, M, m=m, rtol=1e-30, maxiters=m, record=True)
    h = np.array(info["history"])
    assert np.all(np.diff(h) <= 1e-14)
    # the Givens estimate after the cycle equals the true residual of x
    true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(h[-1] - true) <= 1e-10 * max(true, 1e-30) + 1e-14


def test_residual_is_projection_of_r0():
    # proof of Theorem 1: r_m = r0 - Q_m Q_m^T r0 with Q_m the thin Q of A Z_m
    A = I.convdiff2d(7, 100.0).to_scipy()
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    M = _gnp_op(A, L=2, seed=3)
    x, info = K.fgmres(A, b, M, m=8, rtol=1e-30, maxiters=8, record=True)
    Z = info["cycles"][0]["Z"]
    Q, _ = np.linalg.qr(A @ Z)
    r_expected = b - Q @ (Q.T @ b)
    np.testing.assert_allclose(b - A @ x, r_expected, rtol=0, atol=1e-11 * np.linalg.norm(b))


def test_small_system_solved_in_n_steps_with_nonlinear_M():
    # x_m in x0 + span Z_m: with m = n and span Z_n = R^n the residual is zero
    A = I.convdiff2d(5, 10.0).to_scipy()   # n = 25
    n = A.shape[0]
    b = np.random.default_rng(4).standard_normal(n)
    M = _gnp_op(A, L=2, seed=4)
    x, info = K.fgmres(A, b, M, m=n, rtol=1e-11, maxiters=n, record=True)
    assert info["status"] == K.OK
    assert info["iters"] <= n
    assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)


def test_exact_inverse_converges_in_one_step():
    A = I.convdiff2d(6, 100.0).to_scipy()
    Ad = A.toarray()
    b = np.random.default_rng(5).standard_normal(A.shape[0])
    x, info = K.fgmres(A, b, lambda v: np.linalg.solve(Ad, v), m=10, rtol=1e-10, maxiters=50)
    assert info["status"] == K.OK and info["iters"] == 1
    np.testing.assert_allclose(x, np.linalg.solve(Ad, b), rtol=1e-10)


def test_dead_preconditioner_stagnates():
    # M(v) = 0 (all ReLUs dead) gives z = 0: every column is dropped, no progress
    A = I.poisson2d(5).to_scipy()
    b = np.ones(A.shape[0])
    x, info = K.fgmres(A, b, lambda v: np.zeros_like(v), m=5, rtol=1e-8, maxiters=50)
    assert info["status"] == K.STAGNATION
    assert np.all(x == 0)


def test_zero_rhs_and_nan_rhs():
    A = I.poisson2d(4).to_scipy()
    x, info = K.fgmres(A, np.zeros(16), None, m=4)
    assert info["status"] == K.OK and np.all(x == 0) and info["iters"] == 0
    b = np.ones(16)
    b[3] = np.nan
    _, info = K.fgmres(A, b, None, m=4)
    assert info["status"] == K.NAN


def test_not_converged_status_and_iteration_cap():
    A = I.convdiff2d(12, 100.0).to_scipy()
    b = np.random.default_rng(6).standard_normal(A.shape[0])
    _, info = K.fgmres(A, b, None, m=5, rtol=1e-14, maxiters=13)
    assert info["status"] == K.NOT_CONVERGED and info["iters"] == 13
    assert len(info["history"]) == 14


def test_givens_convention():
    c, s, r = K.givens(3.0, 4.0)
    assert (c, s, r) == (0.6, 0.8, 5.0)
    assert K.givens(0.0, 0.0) == (1.0, 0.0, 0.0)
    assert K.givens(-2.0, 0.0) == (-1.0, 0.0, 2.0)


# ------------------------------------------------------------ Eq. 4 / Eq. 5 sampler

def test_arnoldi_unpreconditioned_relation():
    A = I.aniso3d(5, 100.0).to_scipy()
    v1 = K.arnoldi_v1(A.shape[0], seed=7)
    V, H = K.arnoldi(A, v1, 20)
    assert np.linalg.norm(A @ V[:, :-1] - V @ H) <= 1e-12 * np.linalg.norm(H)
    assert np.abs(V.T @ V - np.eye(V.shape[1])).max() <= 1e-12


def test_sampler_algebra():
    # x = V_m Z S^-1 eps  ->  b = A x = V_{m+1} W eps, so ||b|| = ||eps|| and
    # H_bar Q has orthonormal columns (= W); x lies in range(V_m)
    A = I.convdiff2d(9, 100.0).to_scipy()
    V, H = K.arnoldi(A, K.arnoldi_v1(A.shape[0], seed=1), 15)
    Q, s = K.sampler_matrix(H)
    np.testing.assert_allclose((H @ Q).T @ (H @ Q), np.eye(15), atol=1e-10)
    np.testing.assert_allclose(s, np.linalg.svd(H, compute_uv=False), rtol=1e-12)
    X = K.training_x(V, Q, n_arnoldi=4, n_gauss=4, seed=3, step=5)
    eps = PH.normal(15 * 4, 3, 5, PH.STREAM_EPS).reshape(15, 4)
    Bx = A @ X[:, :4]
    np.testing.assert_allclose(np.linalg.norm(Bx, axis=0), np.linalg.norm(eps, axis=0), rtol=1e-9)
    Vm = V[:, :15]
    resid = X[:, :4] - Vm @ (Vm.T @ X[:, :4])
    assert np.linalg.norm(resid) <= 1e-10 * np.linalg.norm(X[:, :4])
    # canonical sign: largest-magnitude entry of each right singular vector is positive
    Z = Q * s[None, :]
    assert np.all(Z[np.argmax(np.abs(Z), axis=0), np.arange(15)] > 0)


def test_cgs2_keeps_orthogonality_under_cancellation():
    # w nearly in span(V): one classical Gram-Schmidt pass leaves components of size
    # eps*||w|| / ||w_out|| along V; the second pass ("twice is enough", Kahan-Parlett)
    # restores orthogonality to working precision.
    rng = np.random.default_rng(8)
    V, _ = np.linalg.qr(rng.standard_normal((200, 6)))
    c = rng.standard_normal(6)
    u = rng.standard_normal(200)
    u -= V @ (V.T @ u)
    u /= np.linalg.norm(u)
    w = V @ c + 1e-9 * u
    h, wo = K.orthogonalise(V, w, "cgs2")
    assert np.abs(V.T @ wo).max() <= 1e-12 * np.linalg.norm(wo)
    np.testing.assert_allclose(h, c, rtol=1e-12)
    assert abs(np.linalg.norm(wo) - 1e-9) <= 1e-6 * 1e-9


def test_pythagorean_subdiagonal_equals_explicit_norm():
    # The CUDA solver takes h_{j+1,j} = ||w1 - V h2|| as sqrt(||w1||^2 - ||h2||^2) with
    # ||w1||^2 from its second-pass reduction.  Against the oracle's explicit norm of the
    # CGS2 output, across cancellation levels down to 1e-10 ||w||, the two agree to a
    # few units of rounding: V is orthonormal to working precision and ||h2|| is
    # O(eps ||w||) after the first pass, so the subtraction cancels nothing.  A sign slip
    # (adding ||h2||^2) or using ||w||^2 instead of ||w1||^2 fails at once.
    rng = np.random.default_rng(29)
    V, _ = np.linalg.qr(rng.standard_normal((500, 20)))
    for delta in (1.0, 1e-3, 1e-6, 1e-8, 1e-10):
        c = rng.standard_normal(20)
        u = rng.standard_normal(500)
        u -= V @ (V.T @ u)
        u /= np.linalg.norm(u)
        w = V @ c + delta * u
        h1 = V.T @ w
        w1 = w - V @ h1
        h2 = V.T @ w1
        explicit = np.linalg.norm(w1 - V @ h2)
        _, wo = K.orthogonalise(V, w, "cgs2")
        assert explicit == np.linalg.norm(wo)  # the oracle's CGS2 output, same operations
        pyth = np.sqrt(max(w1 @ w1 - h2 @ h2, 0.0))
        assert abs(pyth - explicit) <= 8 * np.finfo(float).eps * explicit, (delta, pyth, explicit)
        wrong = np.sqrt(w1 @ w1 + h2 @ h2)
        if delta <= 1e-10:  # ||h2|| is no longer negligible against ||w1|| there
            assert abs(wrong - explicit) > 8 * np.finfo(float).eps * explicit
        wrong_w = np.sqrt(max(w @ w - h2 @ h2, 0.0))
        assert abs(wrong_w - explicit) > 1e-3 * explicit
