"""Parity at the benchmark sizes, in the launch configurations bench.py and apply_bench.py
time (256-row Res-GCONV tiles spread over every block slot, the captured FGMRES cycle).

* The 256 x 256 convection-diffusion matrix (n = 65,536): the whole GNP apply against the
  oracle (float32 1e-5, bfloat16 2e-2); 60 steps of FGMRES(30) with M = I against the
  oracle's residual history (1e-10).
* The 2^20-row power-law matrix: the whole float32 GNP apply against the oracle (1e-5),
  and 2048 sampled rows of one Res-GCONV layer computed one by one from the oracle's
  definition (Eq. 7) on the GPU's own input block.
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def convdiff256():
    A, _ = I.workload("convdiff256")
    return A


@pytest.mark.parametrize("hprec,tol", [(0, 1e-5), (1, 2e-2)])
def test_apply_convdiff256(gnp, convdiff256, hprec, tol):
    import torch
    A = convdiff256
    L = 8
    blob = I.init_weights(L, seed=3)
    blob[32:64] = np.random.default_rng(2).standard_normal(32) * 0.2
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=L, hprec=hprec), blob)
    v = I.gaussian(A.n, seed=9)
    z = torch.empty(A.n, dtype=torch.float32, device="cuda")
    gnp.gnp_apply(M, torch.from_numpy(v).cuda(), z)
    zr = G.forward(G.normalise(A.to_scipy()), v, G.unpack(blob, L), 0)
    assert rel(z.cpu().numpy().astype(np.float64), zr) <= tol


def test_fgmres_identity_convdiff256(gnp, convdiff256):
    import torch
    A = convdiff256
    b = I.spmv(A, np.ones(A.n))
    Mt = gnp.mat_from_csr(A)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = gnp.fgmres_solve(Mt, torch.from_numpy(b).cuda(), x, None, restart=30, rtol=1e-30, maxiters=60)
    _, ir = K.fgmres(A.to_scipy(), b, None, m=30, rtol=1e-30, maxiters=60)
    np.testing.assert_allclose(info.history, ir["history"], rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("tma", ["0", "1"])
def test_apply_and_sampled_layer_powerlaw1m(gnp, tma, monkeypatch):
    """The float32 apply on the 2^20-row power-law matrix within 1e-5 of the oracle, and one
    layer's 2,048 sampled rows from the GPU's own H^0; tma = 1: the TMA-gather kernel."""
    import torch
    monkeypatch.setenv("GNP_GCONV_TMA", tma)
    A, _ = I.workload("powerlaw1m")
    L = 8
    blob = I.init_weights(L, seed=4)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=L), blob)
    v = I.gaussian(A.n, seed=11)
    z = torch.empty(A.n, dtype=torch.float32, device="cuda")
    gnp.gnp_apply(M, torch.from_numpy(v).cuda(), z)
    Ahat = G.normalise(A.to_scipy())
    P = G.unpack(blob, L)
    zr = G.forward(Ahat, v, P, 0)
    assert rel(z.cpu().numpy().astype(np.float64), zr) <= 1e-5
    # one layer, sampled rows: H1_i = ReLU(H0_i U + (A_hat H0)_i W) from the GPU's own H0
    hid = torch.empty((L + 1) * A.n * 16, dtype=torch.float32, device="cuda")
    gnp.gnp_apply_trace(M, torch.from_numpy(v).cuda(), z, hid)
    H = hid.view(L + 1, A.n, 16)
    H0 = H[0].cpu().numpy().astype(np.float64)
    H1 = H[1].cpu().numpy().astype(np.float64)
    rows = np.random.default_rng(0).choice(A.n, 2048, replace=False)
    U, W = P["U"][0], P["W"][0]
    for i in rows:
        s, e = Ahat.indptr[i], Ahat.indptr[i + 1]
        agg = Ahat.data[s:e] @ H0[Ahat.indices[s:e]]
        ref = np.maximum(H0[i] @ U + agg @ W, 0.0)
        assert np.linalg.norm(H1[i] - ref) <= 1e-5 * max(np.linalg.norm(ref), 1e-3), i
    assert gnp.gnp_kernel_faults(reset=True) == 0


@pytest.mark.parametrize("tma", ["0", "1"])
def test_apply_bf16_powerlaw1m(gnp, tma, monkeypatch):
    """The bfloat16 hidden block on the 2^20-row power-law matrix: within 2e-2 of the
    float64 oracle, and much closer to the oracle's bfloat16-store emulation (reading c18),
    which rounds the same stored blocks; tma = 1: the TMA-gather kernel."""
    import torch
    monkeypatch.setenv("GNP_GCONV_TMA", tma)
    A, _ = I.workload("powerlaw1m")
    L = 8
    blob = I.init_weights(L, seed=4)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=L, hprec=1), blob)
    v = I.gaussian(A.n, seed=11)
    z = torch.empty(A.n, dtype=torch.float32, device="cuda")
    gnp.gnp_apply(M, torch.from_numpy(v).cuda(), z)
    zg = z.cpu().numpy().astype(np.float64)
    Ahat = G.normalise(A.to_scipy())
    P = G.unpack(blob, L)
    z64 = G.forward(Ahat, v, P, 0)
    zb = G.forward(Ahat, v, P, 0, hstore="bf16")
    assert rel(zg, z64) <= 2e-2, rel(zg, z64)
    assert rel(zg, zb) <= 0.25 * rel(zg, z64), (rel(zg, zb), rel(zg, z64))
    assert gnp.gnp_kernel_faults(reset=True) == 0
