"""Oracle for flexible GMRES with a nonlinear preconditioner (Sec. 2.1, Eq. 1,
Algorithm 1), the unpreconditioned Arnoldi process (Eq. 4) and the training-pair
sampler built on it (Eq. 5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain float64 numpy.

Readings of the paper taken here (where Algorithm 1 is silent):
* x0 = 0 unless given (Sec. 3 "Problems");
* tol = rtol * ||b||_2 (relative, Sec. 3 "Stopping criteria");
* one *iteration* = one Arnoldi step (one application of M); maxiters counts them;
* inside a cycle the least-squares residual |g_{j+1}| of the Givens QR of H_bar_j
  (Sec. 4 "How robust is GNP?") is checked after every step; when it is <= tol, or
  maxiters is reached, the cycle ends early; x_m is then formed and the true residual
  ||b - A x_m|| decides (the exit test of Algorithm 1);
* Givens: rho = hypot(a, b), c = a/rho, s = b/rho; rho = 0 gives c = 1, s = 0;
* happy breakdown: h_{j+1,j} <= 1e-14 ||A z_j|| ends the cycle keeping column j;
  a rotated diagonal rho <= 1e-14 ||A z_j|| drops column j and ends the cycle;
* two consecutive cycles whose true residual does not decrease -> STAGNATION;
  three consecutive cycles whose Givens estimate met tol while the true residual did
  not -> RESIDUAL_MISMATCH (the "solution failure" of Sec. 4); a NaN -> NAN.
* orthogonalisation: 'mgs' is the loop of Algorithm 1; 'cgs2' is classical
  Gram-Schmidt applied twice (h = h1 + h2), the form the CUDA path uses.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import philox_ref

OK, INVALID_ARG, INVALID_CSR, OOM, CUDA, BREAKDOWN, STAGNATION, RESIDUAL_MISMATCH, \
    NOT_CONVERGED, TIMEOUT, NAN = range(11)

BREAKDOWN_REL = 1e-14


def givens(a: float, b: float):
    """Rotation (c, s, rho) with [c s; -s c] [a; b] = [rho; 0]."""
    rho = float(np.hypot(a, b))
    if rho == 0.0:
        return 1.0, 0.0, 0.0
    return a / rho, b / rho, rho


def orthogonalise(V: np.ndarray, w: np.ndarray, mode: str):
    """Orthogonalise w against the columns of V; returns (h, w_out)."""
    k = V.shape[1]
    if mode == "mgs":
        h = np.zeros(k)
        w = w.copy()
        for i in range(k):
            h[i] = w @ V[:, i]
            w = w - h[i] * V[:, i]
        return h, w
    if mode == "cgs2":
        # second projection is subtracted from the first-pass vector w1, not from w:
        # only then is the output orthogonal to working precision relative to its norm
        h1 = V.T @ w
        w1 = w - V @ h1
        h2 = V.T @ w1
        return h1 + h2, w1 - V @ h2
    raise ValueError(mode)


def fgmres(A, b, M=None, m=30, rtol=1e-8, maxiters=1000, x0=None, orth="cgs2",
           record=False):
    """Restarted FGMRES(m) for A x = b with a (possibly nonlinear) operator M.

    ``M`` maps a float64 vector to a vector (None = identity).  Returns (x, info) where
    info has: status, iters, restarts, history (relative residual after each
    iteration, history[0] = ||r0||/||b||), true_history (true relative residual at the
    start and after every cycle), and with record=True the per-cycle (V, Z, Hbar, beta).
    """
    A = sp.csr_matrix(A)
    n = A.shape[0]
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    Mop = (lambda v: v.copy()) if M is None else M
    bnorm = float(np.linalg.norm(b))
    info = dict(status=OK, iters=0, restarts=0, history=[], true_history=[], cycles=[])
    if bnorm == 0.0:
        x[:] = 0.0
        info["history"] = [0.0]
        info["true_history"] = [0.0]
        return x, info
    tol = rtol * bnorm
    r = b - A @ x
    beta = float(np.linalg.norm(r))
    info["history"].append(beta / bnorm)
    info["true_history"].append(beta / bnorm)
    if not np.isfinite(beta):
        info["status"] = NAN
        return x, info
    if beta <= tol:
        return x, info
    iters = 0
    stagn = 0
    mism = 0
    cycle = 0
    while iters < maxiters:
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        H = np.zeros((m + 1, m))
        R = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        jj = 0
        est_conv = False
        nan = False
        for j in range(m):
            z = Mop(V[:, j])
            Z[:, j] = z
            w = A @ z
            wnorm0 = float(np.linalg.norm(w))
            h, w = orthogonalise(V[:, :j + 1], w, orth)
            hn = float(np.linalg.norm(w))
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0.0:
                V[:, j + 1] = w / hn
            col = H[:j + 2, j].copy()
            for i in range(j):
                t = cs[i] * col[i] + sn[i] * col[i + 1]
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1]
                col[i] = t
            c, s, rho = givens(col[j], col[j + 1])
            iters += 1
            if not (np.isfinite(hn) and np.isfinite(rho) and np.all(np.isfinite(col))):
                nan = True
                jj = j
                break
            if rho <= BREAKDOWN_REL * wnorm0:
                # z_j adds no new direction: drop column j (g untouched), end the cycle
                info["history"].append(abs(g[j]) / bnorm)
                jj = j
                break
            cs[j], sn[j] = c, s
            col[j] = rho
            col[j + 1] = 0.0
            R[:j + 2, j] = col
            g[j + 1] = -s * g[j]
            g[j] = c * g[j]
            jj = j + 1
            res_est = abs(g[j + 1])
            info["history"].append(res_est / bnorm)
            if hn <= BREAKDOWN_REL * wnorm0:
                break
            if res_est <= tol:
                est_conv = True
                break
            if iters >= maxiters:
                break
        if nan:
            info["status"] = NAN
            info["iters"] = iters
            return x, info
        if jj > 0:
            y = np.zeros(jj)
            for i in reversed(range(jj)):
                y[i] = (g[i] - R[i, i + 1:jj] @ y[i + 1:jj]) / R[i, i]
            x = x + Z[:, :jj] @ y
        if record:
            info["cycles"].append(dict(V=V[:, :jj + 1].copy(), Z=Z[:, :jj].copy(),
                                       Hbar=H[:jj + 1, :jj].copy(), beta=beta, jj=jj))
        r = b - A @ x
        beta_new = float(np.linalg.norm(r))
        info["true_history"].append(beta_new / bnorm)
        cycle += 1
        if not np.isfinite(beta_new):
            info["status"] = NAN
            break
        if beta_new <= tol:
            beta = beta_new
            info["status"] = OK
            break
        mism = mism + 1 if est_conv else 0
        stagn = stagn + 1 if beta_new >= beta else 0
        beta = beta_new
        if mism >= 3:
            info["status"] = RESIDUAL_MISMATCH
            break
        if stagn >= 2:
            info["status"] = STAGNATION
            break
        info["restarts"] += 1
        if iters >= maxiters:
            info["status"] = NOT_CONVERGED
            break
    else:
        if beta > tol:
            info["status"] = NOT_CONVERGED
    info["iters"] = iters
    info["final_rel_res"] = beta / bnorm
    return x, info


def gmres_textbook(A, b, m, maxiters, x0=None):
    """Restarted GMRES(m) written the textbook way, for pinning FGMRES with M = I.

    Each step solves min_y ||beta e1 - H_bar_j y|| with a dense least-squares routine
    (no Givens), and the cycle's iterate is x0 + V_m y.  Returns the list of relative
    residual norms after every iteration (index 0 = the initial residual); no early
    exit, so it always runs ``maxiters`` steps (cycles of m).
    """
    A = sp.csr_matrix(A)
    n = A.shape[0]
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    bnorm = np.linalg.norm(b)
    r = b - A @ x
    hist = [np.linalg.norm(r) / bnorm]
    it = 0
    while it < maxiters:
        beta = np.linalg.norm(r)
        V = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        V[:, 0] = r / beta
        y = None
        k = 0
        for j in range(m):
            w = A @ V[:, j]
            for i in range(j + 1):
                H[i, j] = w @ V[:, i]
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
            hist.append(np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y) / bnorm)
            it += 1
            k = j + 1
            if it >= maxiters:
                break
            V[:, j + 1] = w / H[j + 1, j]
        x = x + V[:, :k] @ y
        r = b - A @ x
    return x, hist


# ------------------------------------------------------------- Eq. 4 / Eq. 5 sampler

def arnoldi(A, v1: np.ndarray, m: int):
    """m-step Arnoldi without preconditioner: A V_m = V_{m+1} H_bar_m (Eq. 4), CGS2.

    Stops early at a breakdown h_{j+1,j} <= 1e-14 ||A v_j|| and returns the truncated
    (V_{k+1}, H_bar_k).
    """
    A = sp.csr_matrix(A)
    n = A.shape[0]
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = v1 / np.linalg.norm(v1)
    k = m
    for j in range(m):
        w = A @ V[:, j]
        wn0 = np.linalg.norm(w)
        h, w = orthogonalise(V[:, :j + 1], w, "cgs2")
        H[:j + 1, j] = h
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= BREAKDOWN_REL * wn0:
            k = j + 1
            break
        V[:, j + 1] = w / H[j + 1, j]
    return V[:, :k + 1], H[:k + 1, :k]


def sampler_matrix(Hbar: np.ndarray, rel_cut: float = 1e-14):
    """Q = Z S^{-1} from the SVD H_bar = W S Z^T (Eq. 5), with a canonical form:
    singular values in descending order, each right singular vector signed so that its
    largest-magnitude entry is positive, and 1/s set to 0 for s < rel_cut * s_max."""
    _, s, Zt = np.linalg.svd(Hbar, full_matrices=False)
    Z = Zt.T.copy()
    for k in range(Z.shape[1]):
        i = int(np.argmax(np.abs(Z[:, k])))
        if Z[i, k] < 0:
            Z[:, k] = -Z[:, k]
    inv = np.where(s >= rel_cut * s[0], 1.0 / np.where(s > 0, s, 1.0), 0.0)
    return Z * inv[None, :], s


def arnoldi_v1(n: int, seed: int) -> np.ndarray:
    """Start vector of the sampler's Arnoldi run: Philox stream 3, step 0, normalised."""
    g = philox_ref.normal(n, seed, 0, philox_ref.STREAM_V1)
    return g / np.linalg.norm(g)


def training_x(V: np.ndarray, Q: np.ndarray, n_arnoldi: int, n_gauss: int, seed: int,
               step: int) -> np.ndarray:
    """Solutions x [n, B] of one training batch (Sec. 3: half Eq. 5, half N(0, I_n)).

    Columns 0..n_arnoldi-1: x = V_m Q eps, eps [m, n_arnoldi] from stream 2 (element
    (j, k) at index j*n_arnoldi + k).  Columns n_arnoldi..: x ~ N(0, I) from stream 1
    (element (i, k) at index i*n_gauss + k).
    """
    n = V.shape[0]
    mA = Q.shape[0]
    eps = philox_ref.normal(mA * n_arnoldi, seed, step, philox_ref.STREAM_EPS).reshape(mA, n_arnoldi)
    xa = V[:, :mA] @ (Q @ eps)
    xg = philox_ref.normal(n * n_gauss, seed, step, philox_ref.STREAM_X).reshape(n, n_gauss)
    return np.concatenate([xa, xg], axis=1)
