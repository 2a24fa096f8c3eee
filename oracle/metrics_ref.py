"""Oracle for the paper's convergence metrics (Sec. 3 "Evaluation metrics").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain float64 Python.

* Iter-AUC: the sum over the iterations i = 0..iters of how many decades the relative
  residual r_i = ||b - A x_i|| / ||b|| still lies above rtol.
* Time-AUC: the integral over the solve's elapsed time of the same excess, with r(t)
  constant between iterations; the paper's right-endpoint form takes, for i = 1..iters,
  the excess at iteration i times the time iteration i took, t_i - t_{i-1}.

Reading taken here: a residual of exactly zero (or below the smallest normal double)
counts as 2.2250738585072014e-308, so both metrics stay finite.
"""
from __future__ import annotations

import math

DBL_MIN = 2.2250738585072014e-308


def _excess(r: float, rtol: float) -> float:
    return math.log10(max(r, DBL_MIN)) - math.log10(rtol)


def iter_auc(history, rtol: float) -> float:
    """Iter-AUC of the residual history r_0..r_iters."""
    if rtol <= 0.0 or len(history) < 1:
        return math.nan
    total = 0.0
    for r in history:
        total += _excess(float(r), rtol)
    return total


def time_auc(history, times, rtol: float) -> float:
    """Time-AUC of the residual history r_0..r_iters observed at times t_0..t_iters."""
    if rtol <= 0.0 or len(history) < 1 or len(times) != len(history):
        return math.nan
    total = 0.0
    for i in range(1, len(history)):
        total += _excess(float(history[i]), rtol) * (float(times[i]) - float(times[i - 1]))
    return total
