"""Per-iteration device times, the time limit of fgmres_solve_timeout and the
convergence metrics (Sec. 3 "Stopping criteria", "Evaluation metrics") on the GPU.

* The paper's test problem (x = 1, x0 = 0, rtol 1e-8, maxiters 100): the GPU residual
  history gives the oracle's Iter-AUC (the histories agree to 1e-10); the times are
  non-decreasing, start at >= 0 and end within the host-measured solve time.
* A time limit ends the solve at the first iteration that ends at or after it
  (t_{k-1} < T <= t_k) with GNP_ERR_TIMEOUT, and the result is bit-identical to a solve
  capped at the same k iterations by maxiters (the limit only ends the cycle early).
* A huge limit changes nothing; a negative one is rejected.
"""
import math

import numpy as np
import pytest

from oracle import krylov_ref as K
from oracle import metrics_ref
from paper_2406_00809_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gnp():
    import torch
    from paper_2406_00809_gb300 import build, gnp as g
    build.build()
    assert torch.cuda.is_available()
    return g


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.parametrize("kind", ["poisson", "convdiff"])
def test_paper_protocol_iter_auc_matches_oracle(gnp, kind):
    import torch
    A = I.poisson2d(32) if kind == "poisson" else I.convdiff2d(32, 100.0)
    b = I.spmv(A, np.ones(A.n))
    Mt = gnp.mat_from_csr(A)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = gnp.fgmres_solve(Mt, dev(b), x, None, restart=10, rtol=1e-8, maxiters=100, times=True)
    _, ir = K.fgmres(A.to_scipy(), b, None, m=10, rtol=1e-8, maxiters=100)
    h = np.asarray(ir["history"])
    assert info.iters == ir["iters"] and info.status == ir["status"]
    np.testing.assert_allclose(info.history, h, rtol=1e-10, atol=1e-14)
    assert gnp.iter_auc(info.history, 1e-8) == pytest.approx(metrics_ref.iter_auc(h, 1e-8), abs=1e-7)
    t = info.times
    assert len(t) == len(info.history)
    assert t[0] >= 0.0 and np.all(np.diff(t) >= 0.0) and t[-1] <= info.seconds
    assert t[-1] > 0.0
    assert gnp.time_auc(info.history, t, 1e-8) == pytest.approx(
        metrics_ref.time_auc(info.history, t, 1e-8), rel=1e-12)


def test_timeout_stops_at_the_first_iteration_past_the_limit(gnp):
    import torch
    A = I.convdiff2d(64, 100.0)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=4), I.init_weights(4, seed=1))
    b = dev(I.spmv(A, np.ones(A.n)))
    T = 0.02
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = gnp.fgmres_solve(Mt, b, x, M, restart=30, rtol=1e-30, maxiters=200000, timeout=T, times=True)
    assert info.status == 9, info.status_name  # GNP_ERR_TIMEOUT
    k = info.iters
    assert k >= 2
    assert info.times[k - 1] < T <= info.times[k]
    # the same k steps capped by maxiters: identical iterates, NOT_CONVERGED
    x2 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info2 = gnp.fgmres_solve(Mt, b, x2, M, restart=30, rtol=1e-30, maxiters=k)
    assert info2.status == 8 and info2.iters == k
    assert np.array_equal(info.history, info2.history)
    assert torch.equal(x, x2)
    assert info.rel_res_true == info2.rel_res_true
    # the smallest limit: one step
    x.zero_()
    info = gnp.fgmres_solve(Mt, b, x, M, restart=30, rtol=1e-30, maxiters=100, timeout=1e-9)
    assert info.status == 9 and info.iters == 1


def test_large_timeout_changes_nothing_and_bad_timeout_fails(gnp):
    import torch
    A = I.poisson2d(24)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=2), I.init_weights(2, seed=2))
    b = dev(I.spmv(A, np.ones(A.n)))
    x1 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    x2 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    i1 = gnp.fgmres_solve(Mt, b, x1, M, restart=10, rtol=1e-8, maxiters=300)
    i2 = gnp.fgmres_solve(Mt, b, x2, M, restart=10, rtol=1e-8, maxiters=300, timeout=1e3)
    assert i1.status == i2.status and i1.iters == i2.iters
    assert np.array_equal(i1.history, i2.history) and torch.equal(x1, x2)
    with pytest.raises(gnp.GnpError) as ei:
        gnp.fgmres_solve(Mt, b, x2, M, restart=10, rtol=1e-8, maxiters=300, timeout=-1.0, check=True)
    assert ei.value.status == 1


def test_protocol_runs_all_preconditioners(gnp, capsys):
    """The Sec. 3 protocol script end to end on a small problem: every preconditioner
    reports both runs; the time-limited run ends within one iteration of the limit or
    converges; the GNP's construction time is reported."""
    from paper_2406_00809_gb300 import protocol
    out = protocol.main(["--problems", "poisson32", "--train-steps", "30"])
    run1, run2 = out["poisson32"]
    assert set(run1) == set(run2) == {"none", "jacobi", "gmres", "gnp"}
    limit = max(r["time_s"] for r in run1.values())
    for p in run1:
        assert run1[p]["status"] in ("GNP_OK", "GNP_ERR_NOT_CONVERGED")
        assert run1[p]["iters"] <= 100 and math.isfinite(run1[p]["iter_auc"])
        assert run2[p]["status"] in ("GNP_OK", "GNP_ERR_TIMEOUT")
        if run2[p]["status"] == "GNP_OK":
            assert run2[p]["rel_res"] <= 1e-8
    # Poisson 32^2 with x = 1 converges with inner GMRES within 100 outer steps
    assert run1["gmres"]["status"] == "GNP_OK" and run1["gmres"]["x_err"] < 1e-5
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 5
