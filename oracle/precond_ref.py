"""Oracle for the simple preconditioners the paper compares the GNP with (Sec. 3
"Compared methods"): Jacobi and GMRES used as a preconditioner (inner GMRES).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain float64 numpy.

Readings taken here:
* Jacobi: z_i = v_i / a_ii; a row whose diagonal is zero or not stored passes v_i
  through (z_i = v_i).
* Inner GMRES (the paper: 10 iterations, stopped at relative residual 1e-6): one GMRES
  cycle from z0 = 0 without restart.  Its result is written here from the definition of
  GMRES rather than from Givens rotations: z is the element of the Krylov space
  K_k(A, v) with the smallest residual ||v - A z||, where k is the first step count
  (1..iters) at which that smallest residual is <= rtol ||v||, or iters if none is; an
  Arnoldi breakdown at step k (K_k invariant under A) ends the search at k.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import krylov_ref


def jacobi_diag_inv(A) -> np.ndarray:
    """1 / a_ii per row (1 where a_ii = 0)."""
    d = sp.csr_matrix(A).diagonal().astype(np.float64)
    out = np.ones_like(d)
    nz = d != 0.0
    out[nz] = 1.0 / d[nz]
    return out


def jacobi(A):
    """The Jacobi preconditioner as an operator v -> D^-1 v."""
    dinv = jacobi_diag_inv(A)
    return lambda v: np.asarray(v, dtype=np.float64) * dinv


def inner_gmres_solve(A, v, iters: int = 10, rtol: float = 1e-6):
    """(z, k, residual norm) of the inner GMRES described in the module docstring."""
    v = np.asarray(v, dtype=np.float64)
    beta = float(np.linalg.norm(v))
    if beta == 0.0:
        return np.zeros_like(v), 0, 0.0
    V, Hbar = krylov_ref.arnoldi(A, v, iters)
    kmax = Hbar.shape[1]
    for k in range(1, kmax + 1):
        rhs = np.zeros(k + 1)
        rhs[0] = beta
        Hk = Hbar[:k + 1, :k]
        y = np.linalg.lstsq(Hk, rhs, rcond=None)[0]
        res = float(np.linalg.norm(rhs - Hk @ y))
        if res <= rtol * beta or k == kmax:
            return V[:, :k] @ y, k, res
    raise AssertionError("unreachable")


def inner_gmres(A, iters: int = 10, rtol: float = 1e-6):
    """Inner GMRES as an operator v -> z."""
    return lambda v: inner_gmres_solve(A, v, iters, rtol)[0]
