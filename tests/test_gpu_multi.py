"""Multi-right-hand-side FGMRES (fgmres_solve_multi) on the GPU against the float64 oracle.

* M = identity: every system's residual history and solution equal the oracle's FGMRES
  on that system alone (1e-10), for k = 1..8 (padded to 2, 4, 8 internally), with systems
  that converge at different iterations, a zero right-hand side and a capped one.
* M = GNP (weights trained by the oracle, tests/golden/): every system's iteration count
  lies within the spread that float32-level changes of the oracle's own z cause on that
  system alone, +-2 (tests/golden/make_iteration_bands.py), and its true residual meets
  rtol.
* Bad arguments are rejected.
"""
import json
import os

import numpy as np
import pytest

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


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_weights():
    return np.load(os.path.join(GOLDEN, "gnp_convdiff64_weights.npy"))


def golden_bands():
    return json.load(open(os.path.join(GOLDEN, "gnp_iteration_bands.json")))


def rhs_set(A, k, seed):
    return I.rhs_set(A, k, seed)


@pytest.mark.parametrize("k", [1, 3, 4, 8])
@pytest.mark.parametrize("name", ["convdiff45", "powerlaw12k", "aniso9"])
@pytest.mark.parametrize("form", [0, 1])
def test_multi_apply_matches_oracle(gnp, k, name, form):
    """The k-system GNP kernels (gather of K*64-byte node blocks, one epilogue thread per
    (node, system), decoder fused) against the oracle's forward, column by column."""
    import torch
    from oracle import gnp_ref as G
    A = {"convdiff45": lambda: I.convdiff2d(45, 100.0), "powerlaw12k": lambda: I.powerlaw(12_289, seed=3),
         "aniso9": lambda: I.aniso3d(9, 100.0)}[name]()
    L = 4
    blob = I.init_weights(L, seed=5)
    blob[32:64] = np.random.default_rng(1).standard_normal(32) * 0.2
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=L, form=form), blob)
    V = np.stack([I.gaussian(A.n, seed=30 + r) * (r + 1) for r in range(k)], axis=1)
    Z = torch.empty((A.n, k), dtype=torch.float32, device="cuda")
    gnp.gnp_apply_multi(M, torch.from_numpy(V).cuda(), Z)
    Zh = Z.cpu().numpy().astype(np.float64)
    Ahat = G.normalise(A.to_scipy())
    P = G.unpack(blob, L)
    for r in range(k):
        zr = G.forward(Ahat, V[:, r], P, form)
        err = np.linalg.norm(Zh[:, r] - zr) / np.linalg.norm(zr)
        assert err <= 1e-5, (r, err)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_identity_matches_oracle_per_system(gnp, k):
    import torch
    A = I.convdiff2d(24, 100.0)
    B = rhs_set(A, k, 10)
    Mt = gnp.mat_from_csr(A)
    Bt = torch.from_numpy(B).cuda()
    X = torch.zeros_like(Bt)
    infos = gnp.fgmres_solve_multi(Mt, Bt, X, None, restart=10, rtol=1e-9, maxiters=150)
    Xh = X.cpu().numpy()
    for r in range(k):
        xr, ir = K.fgmres(A.to_scipy(), B[:, r], None, m=10, rtol=1e-9, maxiters=150)
        assert infos[r].status == ir["status"], r
        assert infos[r].iters == ir["iters"], r
        np.testing.assert_allclose(infos[r].history, ir["history"], rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(Xh[:, r], xr, rtol=0, atol=1e-8 * np.abs(xr).max())


def test_identity_zero_rhs_and_cap(gnp):
    import torch
    A = I.poisson2d(20)
    B = rhs_set(A, 4, 3)
    B[:, 2] = 0.0
    Mt = gnp.mat_from_csr(A)
    X = torch.full((A.n, 4), 0.5, dtype=torch.float64, device="cuda")  # x0 = 0.5 (b = A 1 is not solved by it)
    infos = gnp.fgmres_solve_multi(Mt, torch.from_numpy(B).cuda(), X, None, restart=5, rtol=1e-14, maxiters=7)
    assert infos[2].status == 0 and infos[2].iters == 0
    assert float(X[:, 2].abs().max()) == 0.0
    for r in (0, 1, 3):
        assert infos[r].status == 8 and infos[r].iters == 7  # GNP_ERR_NOT_CONVERGED
        _, ir = K.fgmres(A.to_scipy(), B[:, r], None, m=5, rtol=1e-14, maxiters=7,
                         x0=np.full(A.n, 0.5))
        np.testing.assert_allclose(infos[r].history, ir["history"], rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("ortho", ["cgs2", "dcgs2"])
@pytest.mark.parametrize("k", [2, 4, 8])
def test_gnp_iterations_within_oracle_band_per_system(gnp, k, ortho, monkeypatch):
    """Every system of a k-system GNP solve (oracle-trained weights, 64 x 64 problem,
    FGMRES(20), rtol 1e-8) against the oracle's FGMRES on that system alone: the count
    within the spread that float32-level changes of the oracle's z cause, +-2
    (tests/golden/make_iteration_bands.py), and the true residual meets rtol; under both
    orthogonalisation schedules (CGS2, and the second pass overlapped with the layers)."""
    import torch
    monkeypatch.setenv("GNP_ORTHO", ortho)
    A = I.convdiff2d(64, 100.0)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=8), golden_weights())
    B = I.rhs_set(A, 8, 20)[:, :k].copy()
    X = torch.zeros((A.n, k), dtype=torch.float64, device="cuda")
    infos = gnp.fgmres_solve_multi(Mt, torch.from_numpy(B).cuda(), X, M, restart=20, rtol=1e-8, maxiters=1500)
    As = A.to_scipy()
    bands = golden_bands()
    for r in range(k):
        its = [v["iters"] for v in bands[f"convdiff64_rhs{r}"].values()]
        assert infos[r].status == 0, (r, infos[r].status_name)
        assert min(its) - 2 <= infos[r].iters <= max(its) + 2, (r, infos[r].iters, its)
        res = B[:, r] - As @ X[:, r].cpu().numpy()
        assert np.linalg.norm(res) <= 1e-8 * np.linalg.norm(B[:, r]) * (1 + 1e-6)


def test_bad_arguments(gnp):
    import torch
    A = I.poisson2d(8)
    Mt = gnp.mat_from_csr(A)
    B = torch.ones((A.n, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(gnp.GnpError):
        gnp.fgmres_solve_multi(Mt, B, torch.zeros_like(B), None)  # k = 9 > 8
    B = torch.ones((A.n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(gnp.GnpError):
        gnp.fgmres_solve_multi(Mt, B, torch.zeros_like(B), None, restart=65)
