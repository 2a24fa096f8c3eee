"""Pins of the Iter-AUC / Time-AUC oracle (Sec. 3 "Evaluation metrics") and the
library's host implementation of the same metrics checked against it.

Pins (not re-typings of the formula):
* a residual falling one decade per iteration from 1 to rtol = 1e-8 gives the
  triangle 8 + 7 + ... + 0 = 36 decade-iterations, and with unit time steps the
  Time-AUC is that minus the i = 0 term (36 - 8 = 28);
* Time-AUC equals the integral of the piecewise-constant excess curve, evaluated
  independently on a fine grid (midpoint rule over 2 million points);
* Time-AUC scales linearly with the time unit and is invariant to a shift of the
  clock; Iter-AUC grows by len(history) for every decade rtol is lowered;
* a history stuck at r = 1 for k iterations gives k + 1 times -log10(rtol).
"""
import math

import numpy as np
import pytest

from oracle import krylov_ref, metrics_ref
from paper_2406_00809_gb300 import inputs as I


def test_one_decade_per_iteration_triangle():
    hist = [10.0 ** (-i) for i in range(9)]
    assert metrics_ref.iter_auc(hist, 1e-8) == pytest.approx(36.0, abs=1e-12)
    assert metrics_ref.time_auc(hist, list(range(9)), 1e-8) == pytest.approx(28.0, abs=1e-12)


def test_time_auc_is_the_integral_of_the_step_curve():
    rng = np.random.default_rng(3)
    k = 40
    hist = np.concatenate([[1.0], np.exp(np.cumsum(rng.uniform(-1.2, 0.3, size=k)))])
    t = np.concatenate([[0.0], np.cumsum(rng.uniform(0.01, 0.2, size=k))])
    rtol = 1e-6
    # r(t) = r_i on (t_{i-1}, t_i]; integrate log10 r(t) - log10 rtol on a fine grid
    N = 2_000_000
    grid = (np.arange(N) + 0.5) * (t[-1] / N)
    idx = np.searchsorted(t, grid, side="left")
    f = np.log10(hist[idx]) - math.log10(rtol)
    integral = f.sum() * (t[-1] / N)
    assert metrics_ref.time_auc(hist, t, rtol) == pytest.approx(integral, rel=1e-4)


def test_scaling_and_shift_invariances():
    rng = np.random.default_rng(5)
    hist = np.exp(-np.cumsum(rng.uniform(0, 1, size=20)))
    t = np.cumsum(rng.uniform(0, 1, size=20))
    a = metrics_ref.time_auc(hist, t, 1e-8)
    assert metrics_ref.time_auc(hist, 3.0 * t, 1e-8) == pytest.approx(3.0 * a, rel=1e-12)
    assert metrics_ref.time_auc(hist, t + 7.5, 1e-8) == pytest.approx(a, rel=1e-9)
    i8 = metrics_ref.iter_auc(hist, 1e-8)
    assert metrics_ref.iter_auc(hist, 1e-9) == pytest.approx(i8 + len(hist), rel=1e-12)


def test_stuck_history_and_zero_residual():
    assert metrics_ref.iter_auc([1.0] * 6, 1e-8) == pytest.approx(48.0)
    # an exact zero counts as the smallest normal double: finite
    v = metrics_ref.iter_auc([1.0, 0.0], 1e-8)
    assert math.isfinite(v) and v == pytest.approx(8.0 + (-307.6526555685888 + 8.0), rel=1e-12)
    assert math.isnan(metrics_ref.iter_auc([], 1e-8))
    assert math.isnan(metrics_ref.iter_auc([1.0], 0.0))


@pytest.fixture(scope="module")
def gnp():
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp as g
    return g


def test_library_metrics_match_the_oracle(gnp):
    """Host functions gnp_iter_auc / gnp_time_auc (no device work) on a real FGMRES
    history of the oracle."""
    A = I.poisson2d(16)
    b = I.spmv(A, np.ones(A.n))
    _, info = krylov_ref.fgmres(A.to_scipy(), b, m=10, rtol=1e-8, maxiters=100)
    hist = np.array(info["history"])
    t = np.cumsum(np.r_[0.0, np.full(len(hist) - 1, 1.3e-4)])
    for rtol in (1e-8, 1e-6, 1e-12):
        assert gnp.iter_auc(hist, rtol) == pytest.approx(metrics_ref.iter_auc(hist, rtol), rel=1e-13)
        assert gnp.time_auc(hist, t, rtol) == pytest.approx(metrics_ref.time_auc(hist, t, rtol), rel=1e-13)
    assert gnp.iter_auc(np.array([1.0, 0.0]), 1e-8) == pytest.approx(metrics_ref.iter_auc([1.0, 0.0], 1e-8))
    assert math.isnan(gnp.iter_auc(np.array([1.0]), -1.0))
