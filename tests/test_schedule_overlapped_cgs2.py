"""Pins for reading c32: the overlapped (delayed-reorthogonalisation) CGS2 schedule of the
GNP-preconditioned FGMRES step, written here in float64 numpy in the order the kernels
run it, and checked against what the mathematics of Sec. 2.1 / Algorithm 1 fixes.

Per step s of a cycle (v'_0 = v_0 = r / ||r||):
  z_s = M(v'_s);  for s >= 1: a_s = V_{s-1}^T v'_s, nu_s = sqrt(||v'_s||^2 - ||a_s||^2),
  column s-1 = [h_{s-1} + rho_{s-1} a_s; rho_{s-1} nu_s],  v_s = (v'_s - V_{s-1} a_s) / nu_s;
  w = A z_s,  h_s = V_s^T w,  rho_s = sqrt(||w||^2 - ||h_s||^2),
  v'_{s+1} = (w - V_s h_s) / max(rho_s, 1e-7 ||w||);
the last column of the cycle keeps its first-pass values [h_{m-1}; rho_{m-1}].

Checked: the flexible Arnoldi relation A Z_m = [V_m, v_m'] H_bar (v_m' = (w - V h) / rho of
the last column, which the kernels never form) and the orthonormality of
V_m to rounding; the cycle's least-squares residuals against a CGS2 cycle of the oracle
(oracle/krylov_ref.py) with M = I and with a nonlinear GNP; an exact breakdown ends the
cycle on the right column; the normalisation floor keeps the relation exact when the
Pythagorean rho cancels to 0; and first-pass dot products with an injected error, which
only the lagged correction column and the reorthogonalisation make exact again.
"""
import numpy as np
import pytest

from oracle import gnp_ref as G
from oracle import krylov_ref as K
from paper_2406_00809_gb300 import inputs as I

RHO_FLOOR = 1e-7
BREAKDOWN_REL = 1e-14


def overlapped_cycle(A, r, M, m, rho_floor=RHO_FLOOR, dot_err=0.0, seed=0):
    """One restart cycle in the kernels' order.  Returns (V [m+1, n] with row m = v'_m,
    Z [m, n], Hbar [m+1, m], jj = columns kept, beta).  dot_err > 0 adds a relative error
    of that size to the first-pass dot products h (as a lossy reduction would), which v'
    then carries as components along V_s for the next reorthogonalisation to remove."""
    rng = np.random.default_rng(seed)
    n = r.size
    beta = np.linalg.norm(r)
    V = np.zeros((m + 1, n))
    Z = np.zeros((m, n))
    H = np.zeros((m + 1, m))
    V[0] = r / beta
    hprev = None
    rho_prev = wn_prev = None
    jj = m
    for s in range(m):
        Z[s] = M(V[s]) if M is not None else V[s]
        if s >= 1:
            a = V[:s] @ V[s]
            nu = np.sqrt(max(V[s] @ V[s] - a @ a, 0.0))
            H[:s, s - 1] = hprev + rho_prev * a
            H[s, s - 1] = rho_prev * nu
            if H[s, s - 1] <= BREAKDOWN_REL * wn_prev:  # column s-1 breaks down: the cycle ends
                return V, Z, H, s, beta
            V[s] = (V[s] - a @ V[:s]) / nu
        w = A @ Z[s]
        h = V[:s + 1] @ w
        if dot_err:
            h = h + dot_err * np.linalg.norm(w) * rng.standard_normal(h.size)
        omega = w @ w
        rho = np.sqrt(max(omega - h @ h, 0.0))
        rho_n = max(rho, rho_floor * np.sqrt(omega))
        if s == m - 1:
            # the last column keeps [h; rho] (Pythagorean, unfloored); the kernels never form
            # v'_m, so the vector that goes with it here is the one rho normalises
            H[:s + 1, s] = h
            H[s + 1, s] = rho
            V[s + 1] = (w - h @ V[:s + 1]) / rho
            break
        V[s + 1] = (w - h @ V[:s + 1]) / rho_n
        hprev, rho_prev, wn_prev = h, rho_n, np.sqrt(omega)
    return V, Z, H, jj, beta


def lsq_history(H, beta, cols):
    """||beta e1 - H_bar[:, :j] y_j|| for j = 0..cols (dense least squares)."""
    out = [beta]
    for j in range(1, cols + 1):
        e1 = np.zeros(j + 1)
        e1[0] = beta
        y = np.linalg.lstsq(H[:j + 1, :j], e1, rcond=None)[0]
        out.append(np.linalg.norm(e1 - H[:j + 1, :j] @ y))
    return np.array(out)


def _gnp(A, L=2, seed=0):
    Ahat = G.normalise(A)
    P = G.unpack(I.init_weights(L, seed=seed), L)
    return lambda v: G.forward(Ahat, v, P, 0)


@pytest.mark.parametrize("precond", ["identity", "gnp"])
def test_arnoldi_relation_and_orthonormality(precond):
    A = I.convdiff2d(16, 100.0).to_scipy()
    r = np.random.default_rng(0).standard_normal(A.shape[0])
    M = None if precond == "identity" else _gnp(A)
    m = 30
    V, Z, H, jj, beta = overlapped_cycle(A, r, M, m)
    assert jj == m
    AZ = (A @ Z.T)
    rel = np.linalg.norm(AZ - V.T @ H) / np.linalg.norm(AZ)
    assert rel <= 1e-13, rel
    orth = np.linalg.norm(V[:m] @ V[:m].T - np.eye(m))
    assert orth <= 1e-13, orth
    # the last vector has only the first pass: orthogonal to V_m to single-pass accuracy
    assert np.max(np.abs(V[:m] @ V[m])) <= 1e-8


@pytest.mark.parametrize("precond", ["identity", "gnp"])
def test_residuals_match_a_cgs2_cycle(precond):
    """With exact arithmetic a_s = 0 and nu_s = 1, so the least-squares residuals of the
    cycle equal those of the oracle's CGS2 cycle (one cycle of FGMRES(30), rtol 0)."""
    A = I.convdiff2d(16, 100.0).to_scipy()
    r = np.random.default_rng(1).standard_normal(A.shape[0])
    M = None if precond == "identity" else _gnp(A, seed=2)
    m = 30
    V, Z, H, jj, beta = overlapped_cycle(A, r, M, m)
    hist = lsq_history(H, beta, jj) / beta
    _, info = K.fgmres(A, r, M, m=m, rtol=1e-30, maxiters=m, orth="cgs2")
    ref = np.asarray(info["history"])
    tol = 1e-9 if precond == "identity" else 1e-6
    np.testing.assert_allclose(hist, ref[:jj + 1], rtol=tol)


def test_exact_breakdown_ends_the_cycle():
    """A 16-row system: the Krylov space is exhausted after 16 directions, so a subdiagonal
    reaches the breakdown level, the cycle keeps the columns before it, and those columns
    solve the system exactly."""
    A = I.poisson2d(4).to_scipy()
    r = np.random.default_rng(3).standard_normal(16)
    V, Z, H, jj, beta = overlapped_cycle(A, r, None, 30)
    assert 14 <= jj <= 17, jj
    e1 = np.zeros(jj + 1)
    e1[0] = beta
    y = np.linalg.lstsq(H[:jj + 1, :jj], e1, rcond=None)[0]
    x = Z[:jj].T @ y
    assert np.linalg.norm(r - A @ x) <= 1e-10 * beta


def test_floor_keeps_the_relation_when_rho_cancels():
    """Force the Pythagorean rho to cancel (a floor far above the true rho): v' is then
    normalised by the floor, and nu of the next step restores the true subdiagonal, so
    the relation still holds to rounding."""
    A = I.convdiff2d(12, 100.0).to_scipy()
    r = np.random.default_rng(4).standard_normal(A.shape[0])
    m = 20
    V, Z, H, jj, beta = overlapped_cycle(A, r, None, m, rho_floor=0.5)
    AZ = A @ Z[:jj].T
    rel = np.linalg.norm(AZ - V[:jj + 1].T @ H[:jj + 1, :jj]) / np.linalg.norm(AZ)
    assert rel <= 1e-12, rel
    orth = np.linalg.norm(V[:jj] @ V[:jj].T - np.eye(jj))
    assert orth <= 1e-12, orth


def test_lagged_column_removes_first_pass_errors():
    """First-pass dot products off by 1e-6 (relative): v' then has components of that size
    along V_s, a_s is no longer O(eps), and the Arnoldi relation and the orthonormality of V
    hold to rounding only because column s-1 adds rho_{s-1} a_s and v_s is reorthogonalised."""
    A = I.convdiff2d(16, 100.0).to_scipy()
    r = np.random.default_rng(5).standard_normal(A.shape[0])
    m = 30
    V, Z, H, jj, beta = overlapped_cycle(A, r, _gnp(A, seed=1), m, dot_err=1e-6, seed=6)
    assert jj == m
    AZ = A @ Z.T
    rel = np.linalg.norm(AZ - V.T @ H) / np.linalg.norm(AZ)
    assert rel <= 1e-12, rel
    orth = np.linalg.norm(V[:m] @ V[:m].T - np.eye(m))
    assert orth <= 1e-12, orth
