"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module only *builds problems*: sparse matrices in CSR form (int32 row_ptr/col,
float64 values), right-hand sides and initial weight blobs.  It holds none of the
method's arithmetic (no gamma normalisation, no GNN, no Krylov step).  Both the
oracle and the GPU tests import it so that the two sides see identical inputs.

The paper evaluates on SuiteSparse (square, real, non-SPD, 1K-100K rows, nnz < 2M;
Sec. 3 "Problems").  That collection is not reproduced here; these generators stand
in for it with PDE-like and general sparse matrices of the same shape range and
beyond:

* ``poisson2d``   5-point Laplacian on an nx x nx grid, Dirichlet boundary.
* ``convdiff2d``  -Lap(u) + beta (u_x + u_y) on the unit square, first-order upwind,
                  nonsymmetric.
* ``aniso3d``     7-point -(u_xx + u_yy + eps_z u_zz) on an nx^3 grid.
* ``powerlaw``    general sparse matrix, power-law row lengths, N(0,1) values plus a
                  diagonal shift calibrated to cond ~ 1e6, random symmetric
                  permutation.

Weight blobs follow the layout documented in ``include/gnp.h``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

D_HIDDEN = 16   # Res-GCONV width d (Sec. 3 "Hyperparameters")
MLP_HIDDEN = 32  # encoder/decoder hidden width (Sec. 3 "Hyperparameters")


@dataclass
class CSR:
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            for k in range(self.row_ptr[i], self.row_ptr[i + 1]):
                A[i, self.col[k]] += self.val[k]
        return A


def _from_coo(n, rows, cols, vals) -> CSR:
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr.astype(np.int32), cols.astype(np.int32), vals)


def _stencil(shape, offsets_vals):
    """Assemble a constant-coefficient stencil on a Dirichlet box grid."""
    dims = len(shape)
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    rows, cols, vals = [], [], []
    for off, v in offsets_vals:
        src = [slice(None)] * dims
        dst = [slice(None)] * dims
        for ax, o in enumerate(off):
            if o > 0:
                src[ax] = slice(0, shape[ax] - o)
                dst[ax] = slice(o, shape[ax])
            elif o < 0:
                src[ax] = slice(-o, shape[ax])
                dst[ax] = slice(0, shape[ax] + o)
        r = idx[tuple(src)].ravel()
        c = idx[tuple(dst)].ravel()
        rows.append(r)
        cols.append(c)
        vals.append(np.full(r.shape, v, dtype=np.float64))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def poisson2d(nx: int) -> CSR:
    """5-point Poisson on nx x nx: 4 on the diagonal, -1 for each grid neighbour."""
    offs = [((0, 0), 4.0), ((0, -1), -1.0), ((0, 1), -1.0), ((-1, 0), -1.0), ((1, 0), -1.0)]
    return _stencil((nx, nx), offs)


def convdiff2d(nx: int, beta: float = 100.0) -> CSR:
    """-Lap(u) + beta (u_x + u_y), h = 1/(nx+1), first-order upwind (beta > 0).

    Row stencil: centre 4/h^2 + 2 beta/h; west/south -1/h^2 - beta/h; east/north -1/h^2.
    Grid index = y*nx + x.
    """
    h = 1.0 / (nx + 1)
    c = 4.0 / h**2 + 2.0 * beta / h
    up = -1.0 / h**2 - beta / h
    dn = -1.0 / h**2
    offs = [((0, 0), c), ((0, -1), up), ((-1, 0), up), ((0, 1), dn), ((1, 0), dn)]
    return _stencil((nx, nx), offs)


def aniso3d(nx: int, eps_z: float = 100.0) -> CSR:
    """7-point -(u_xx + u_yy + eps_z u_zz) on nx^3 (index z*nx*nx + y*nx + x)."""
    c = 4.0 + 2.0 * eps_z
    offs = [((0, 0, 0), c),
            ((0, 0, -1), -1.0), ((0, 0, 1), -1.0),
            ((0, -1, 0), -1.0), ((0, 1, 0), -1.0),
            ((-1, 0, 0), -eps_z), ((1, 0, 0), -eps_z)]
    return _stencil((nx, nx, nx), offs)


def powerlaw_exponent(mean: float = 12.0, kmin: int = 2, kmax: int = 2000) -> float:
    """Exponent a of P(k) ~ k^-a on [kmin, kmax] whose mean row length is ``mean`` (bisection)."""
    k = np.arange(kmin, kmax + 1, dtype=np.float64)
    lo, hi = 0.0, 6.0
    for _ in range(200):
        a = 0.5 * (lo + hi)
        p = k ** (-a)
        m = (p * k).sum() / p.sum()
        if m > mean:
            lo = a
        else:
            hi = a
    return 0.5 * (lo + hi)


def _powerlaw_lengths(rng, n: int, mean: float, kmax: int) -> np.ndarray:
    """Row lengths k (diagonal included) drawn from P(k) ~ k^-a on [2, kmax]."""
    k = np.arange(2, kmax + 1)
    a = powerlaw_exponent(mean, 2, kmax)
    p = k.astype(np.float64) ** (-a)
    p /= p.sum()
    return rng.choice(k, size=n, p=p)


def powerlaw_unshifted(n: int, mean: float = 12.0, kmax: int = 2000, seed: int = 0):
    """The random part of the power-law matrix, before the diagonal shift and permutation.

    Returns (rows, cols, vals, diag): the off-diagonal entries in COO form (values
    N(0, 1), columns uniform over the other n - 1 indices, repeated (row, col) pairs
    dropped) and the N(0, 1) diagonal.  The draws consume ``seed``'s PCG64 stream in
    this order: row lengths, columns, off-diagonal values, diagonal values, permutation.
    """
    rng = np.random.default_rng(seed)
    kmax = min(kmax, n)
    lens = _powerlaw_lengths(rng, n, mean, kmax)
    off = lens - 1
    total = int(off.sum())
    rows = np.repeat(np.arange(n, dtype=np.int64), off)
    cols = rng.integers(0, n - 1, size=total, dtype=np.int64)
    cols = cols + (cols >= rows)  # skip the diagonal
    # drop repeated (row, col) pairs: sort the keys once, keep first occurrences
    key = np.sort(rows * n + cols)
    keep = np.ones(key.size, dtype=bool)
    keep[1:] = key[1:] != key[:-1]
    key = key[keep]
    rows = key // n
    cols = key % n
    vals = rng.standard_normal(rows.shape[0])
    diag = rng.standard_normal(n)
    return rows, cols, vals, diag, rng


def powerlaw_radius(vals: np.ndarray, diag: np.ndarray) -> float:
    """Spectral-radius estimate of the unshifted matrix: the root-mean-square row norm
    sqrt(sum a_ij^2 / n), the radius of the circular law for independent entries."""
    n = diag.size
    return float(np.sqrt((np.dot(vals, vals) + np.dot(diag, diag)) / n))


def _powerlaw_shift_fraction() -> float:
    import json
    import os
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "powerlaw_shift.json")
    return float(json.load(open(p))["fraction"])


def powerlaw(n: int, mean: float = 12.0, kmax: int = 2000, shift_fraction: float | None = None,
             seed: int = 0, permute: bool = True) -> CSR:
    """General sparse ill-conditioned matrix with power-law row lengths.

    * row length k (diagonal included) ~ P(k) ~ k^-a on [2, min(kmax, n)], a chosen so
      E[k] = mean;
    * off-diagonal columns uniform without repeats; every value, the diagonal included,
      N(0, 1);
    * a diagonal shift s I with s = shift_fraction * rho, rho the circular-law radius of
      the unshifted matrix (``powerlaw_radius``).  The default fraction is the one that
      ``powerlaw_calibration.py`` found by dense singular values to give cond(A) ~ 1e6
      at n = 4,096 and 16,384 (stored in ``powerlaw_shift.json``);
    * a random symmetric permutation P A P^T (the shift stays on the diagonal).
    """
    rows, cols, vals, diag, rng = powerlaw_unshifted(n, mean, kmax, seed)
    if shift_fraction is None:
        shift_fraction = _powerlaw_shift_fraction()
    s = shift_fraction * powerlaw_radius(vals, diag)
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, diag + s])
    perm = rng.permutation(n) if permute else np.arange(n)
    return _from_coo_fast(n, perm[rows], perm[cols], vals)


def _from_coo_fast(n, rows, cols, vals) -> CSR:
    """CSR from unique (row, col) pairs via one sort of the combined key."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.argsort(rows * n + cols, kind="stable")
    rows, cols, vals = rows[order], cols[order], np.asarray(vals, dtype=np.float64)[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr.astype(np.int32), cols.astype(np.int32), vals)


def gaussian(n: int, seed: int, batch: int | None = None) -> np.ndarray:
    """x ~ N(0, I) as float64, shape [n] or [n, batch] (numpy PCG64 stream ``seed``)."""
    rng = np.random.default_rng(seed)
    if batch is None:
        return rng.standard_normal(n)
    return rng.standard_normal((n, batch))


def rhs_set(A: CSR, k: int, seed: int) -> np.ndarray:
    """k right-hand sides b = A x of different character, as columns of an [n, k] array:
    x = 1 (r % 3 == 0), a smooth sine (r % 3 == 1), x ~ N(0, 1) with seed + r (otherwise)."""
    n = A.n
    cols = []
    for r in range(k):
        if r % 3 == 0:
            x = np.ones(n)
        elif r % 3 == 1:
            x = np.sin(np.linspace(0, 3 * (r + 1), n))
        else:
            x = gaussian(n, seed=seed + r)
        cols.append(spmv(A, x))
    return np.stack(cols, axis=1)


def spmv(A: CSR, x: np.ndarray) -> np.ndarray:
    """b = A x for building right-hand sides from a chosen solution (problem setup only)."""
    return A.to_scipy() @ x


def weight_count(L: int) -> int:
    """Length of the flat weight blob for L Res-GCONV layers (layout in include/gnp.h)."""
    d, hdim = D_HIDDEN, MLP_HIDDEN
    enc = hdim + hdim + hdim * d + d
    lay = 2 * d * d
    dec = d * hdim + hdim + hdim + 1
    return enc + L * lay + dec


def init_weights(L: int, seed: int, gconv_std: float = 0.25) -> np.ndarray:
    """Gaussian initial weights: U_l, W_l ~ N(0, gconv_std^2) (default 1/sqrt(16));
    MLP weights ~ N(0, 1/fan_in); biases 0.  Returned as float32 in blob order."""
    rng = np.random.default_rng(seed)
    d, hdim = D_HIDDEN, MLP_HIDDEN
    parts = [rng.standard_normal(hdim) * 1.0,            # enc W1 (1 x 32), fan_in 1
             np.zeros(hdim),                             # enc b1
             rng.standard_normal(hdim * d) / np.sqrt(hdim),  # enc W2 (32 x 16)
             np.zeros(d)]                                # enc b2
    for _ in range(L):
        parts.append(rng.standard_normal(d * d) * gconv_std)  # U_l
        parts.append(rng.standard_normal(d * d) * gconv_std)  # W_l
    parts += [rng.standard_normal(d * hdim) / np.sqrt(d),    # dec W1 (16 x 32)
              np.zeros(hdim),                                # dec b1
              rng.standard_normal(hdim) / np.sqrt(hdim),     # dec W2 (32 x 1)
              np.zeros(1)]                                   # dec b2
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == weight_count(L)
    return w


# ---------------------------------------------------------------- named workloads

def workload(name: str):
    """Matrix + settings of the named synthetic workloads.

    Returns (CSR, dict of settings).  Names: 'poisson32' (n=1,024), 'convdiff256'
    (n=65,536), 'powerlaw1m' (n=2^20), 'aniso64' (n=262,144) and small variants
    used by tests ('convdiff64', 'powerlaw64k', 'aniso8').
    """
    if name == "poisson32":
        return poisson2d(32), dict(L=4, restart=10, rtol=1e-6, maxiters=200)
    if name == "convdiff256":
        return convdiff2d(256, 100.0), dict(L=8, restart=30, rtol=1e-8, maxiters=1000)
    if name == "convdiff64":
        return convdiff2d(64, 100.0), dict(L=8, restart=30, rtol=1e-8, maxiters=1000)
    if name == "powerlaw1m":
        return powerlaw(1 << 20, seed=0), dict(L=8, restart=50, rtol=1e-8, maxiters=1000)
    if name == "powerlaw64k":
        return powerlaw(1 << 16, seed=0), dict(L=8, restart=50, rtol=1e-8, maxiters=1000)
    if name == "aniso64":
        return aniso3d(64, 100.0), dict(L=8, batch=32, arnoldi_m=30)
    if name == "aniso8":
        return aniso3d(8, 100.0), dict(L=8, batch=32, arnoldi_m=30)
    raise KeyError(name)
