"""The one-reduction CGS2 schedule of the GNP-preconditioned FGMRES step (Sec. 2.1,
Algorithm 1 with delayed reorthogonalisation; GNP_ORTHO=dcgs2) against the oracle and
against the two-reduction CGS2 step, at the edges of its lagged bookkeeping: restart
lengths 1 and 2 (the cycle-end kernel finishes one or two columns), solves that stop
inside a cycle on the residual estimate, and an exact breakdown of the Krylov space (a
16-row system with restart 30).

In exact arithmetic the two schedules take the same steps (the reorthogonalisation
coefficients vanish), so on these well-conditioned problems their residual histories
agree to float32-level noise of the GNP and their statuses are equal.
"""
import numpy as np
import pytest

from oracle import gnp_ref as G
from oracle import krylov_ref as K
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


def solve(gnp, A, blob, L, b, m, rtol, maxit, ortho, monkeypatch):
    import torch
    monkeypatch.setenv("GNP_ORTHO", ortho)
    Mt = gnp.mat_from_csr(A)
    Mg = gnp.gnp_create(Mt, gnp.make_config(L=L), blob)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = gnp.fgmres_solve(Mt, dev(b), x, Mg, restart=m, rtol=rtol, maxiters=maxit)
    return info, x.cpu().numpy()


@pytest.mark.parametrize("m", [1, 2, 5])
def test_short_restarts_match_oracle(gnp, m, monkeypatch):
    """FGMRES(m) for m = 1, 2, 5 with an untrained GNP on the 16 x 16 Poisson matrix: the
    first 8 residuals agree with the float64 oracle to 1e-5, the status and iteration
    count with the CGS2 step's, and the returned x has the reported true residual."""
    A = I.poisson2d(16)
    L = 2
    blob = I.init_weights(L, seed=3)
    b = I.spmv(A, I.gaussian(A.n, seed=1))
    info, x = solve(gnp, A, blob, L, b, m, 1e-30, 40, "dcgs2", monkeypatch)
    ref, _ = solve(gnp, A, blob, L, b, m, 1e-30, 40, "cgs2", monkeypatch)
    M64 = lambda v: G.forward(G.normalise(A.to_scipy()), v, G.unpack(blob, L), 0)  # noqa: E731
    _, ir = K.fgmres(A.to_scipy(), b, M64, m=m, rtol=1e-30, maxiters=40)
    h = np.asarray(ir["history"])
    np.testing.assert_allclose(info.history[:9], h[:9], rtol=1e-5)
    assert info.status == ref.status and info.iters == ref.iters
    r = b - A.to_scipy() @ x
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - info.rel_res_true) <= 1e-10


@pytest.mark.parametrize("rtol", [1e-6, 1e-8])
def test_stop_inside_a_cycle(gnp, rtol, monkeypatch):
    """The oracle-trained weights (tests/golden/gnp_convdiff64_weights.npy) on the 64 x 64
    convection-diffusion matrix with FGMRES(30): the oracle converges inside the first
    cycle (rtol 1e-6) or the second (1e-8).  The solve stops on the residual estimate
    one step after its deciding column in the one-reduction schedule; the count must be
    the oracle's +-2, the status OK and the true residual at rtol."""
    import os
    A = I.convdiff2d(64, 100.0)
    L = 8
    blob = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gnp_convdiff64_weights.npy"))
    b = I.spmv(A, I.gaussian(A.n, seed=0))
    info, x = solve(gnp, A, blob, L, b, 30, rtol, 600, "dcgs2", monkeypatch)
    M64 = lambda v: G.forward(G.normalise(A.to_scipy()), v, G.unpack(blob, L), 0)  # noqa: E731
    _, ir = K.fgmres(A.to_scipy(), b, M64, m=30, rtol=rtol, maxiters=600)
    assert info.status == 0 and ir["status"] == 0, info.status_name
    assert abs(info.iters - ir["iters"]) <= 2, (info.iters, ir["iters"])
    assert info.iters % 30 != 0
    r = b - A.to_scipy() @ x
    assert np.linalg.norm(r) <= rtol * np.linalg.norm(b) * (1 + 1e-9)


@pytest.mark.parametrize("rtol", [1e-12, 1e-30])
def test_exact_breakdown(gnp, rtol, monkeypatch):
    """A 16-row system with FGMRES(30): the Krylov space is exhausted within 16 steps, so
    the subdiagonal reaches the breakdown level and the cycle must end on that column with
    no NaN; x solves the system to 1e-10.  At rtol 1e-12 both schedules converge.  At
    1e-30 both end below rounding, where whether a cycle still lowers the residual is
    noise: each may stop on stagnation or on maxiters."""
    A = I.poisson2d(4)
    L = 2
    blob = I.init_weights(L, seed=5)
    b = I.spmv(A, I.gaussian(A.n, seed=2))
    info, x = solve(gnp, A, blob, L, b, 30, rtol, 90, "dcgs2", monkeypatch)
    ref, xr = solve(gnp, A, blob, L, b, 30, rtol, 90, "cgs2", monkeypatch)
    if rtol == 1e-12:
        assert info.status == ref.status == 0, (info.status_name, ref.status_name)
    else:
        for st in (info.status_name, ref.status_name):
            assert st in ("GNP_ERR_STAGNATION", "GNP_ERR_NOT_CONVERGED"), st
    for xx in (x, xr):
        r = b - A.to_scipy() @ xx
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    assert np.all(np.isfinite(info.history))


@pytest.mark.parametrize("mat", ["poisson16", "powerlaw3000"])
@pytest.mark.parametrize("m", [1, 2, 5])
def test_multi_short_restarts_match_oracle(gnp, m, mat, monkeypatch):
    """The k-system solver (three systems, untrained GNP) on the overlapped schedule with
    restart lengths 1, 2 and 5, on the 16 x 16 Poisson matrix (short-row kernels) and a
    3,000-row power-law matrix with rows of up to 999 nonzeros (tile kernels; shift 1.25 x
    its spectral radius): each system's first 8 residuals agree with the oracle's FGMRES
    on that system alone to 1e-5, and its status and iteration count equal the
    two-reduction k-system solve's."""
    import torch
    A = I.poisson2d(16) if mat == "poisson16" else I.powerlaw(3000, seed=7, shift_fraction=1.25)
    L = 2
    blob = I.init_weights(L, seed=3)
    B = np.stack([I.spmv(A, I.gaussian(A.n, seed=s)) for s in (1, 2, 3)], axis=1)
    Mt = gnp.mat_from_csr(A)
    Mg = gnp.gnp_create(Mt, gnp.make_config(L=L), blob)
    runs = {}
    for ortho in ("dcgs2", "cgs2"):
        monkeypatch.setenv("GNP_ORTHO", ortho)
        X = torch.zeros((A.n, 3), dtype=torch.float64, device="cuda")
        runs[ortho] = gnp.fgmres_solve_multi(Mt, torch.from_numpy(B).cuda(), X, Mg, restart=m, rtol=1e-30,
                                             maxiters=30)
    M64 = lambda v: G.forward(G.normalise(A.to_scipy()), v, G.unpack(blob, L), 0)  # noqa: E731
    for r in range(3):
        _, ir = K.fgmres(A.to_scipy(), B[:, r], M64, m=m, rtol=1e-30, maxiters=30)
        got = runs["dcgs2"][r]
        np.testing.assert_allclose(got.history[:9], np.asarray(ir["history"])[:9], rtol=1e-5)
        assert got.status == runs["cgs2"][r].status and got.iters == runs["cgs2"][r].iters
