"""The Jacobi and inner-GMRES preconditioners and the gnp_precond handle on the GPU,
against the float64 oracle (Sec. 3 "Compared methods").

* gnp_precond_apply: Jacobi bit-exact; inner GMRES (one cycle, stopped at rtol or after
  `iters` steps) to 1e-10 of the oracle's minimal-residual definition.
* FGMRES preconditioned by Jacobi / inner GMRES: residual histories and iteration counts
  agree with the oracle's FGMRES using the oracle's operators (to 1e-9, float64 on both
  sides).
* The identity and GNP kinds through the handle give bit-identical results to
  fgmres_solve with no preconditioner / with the model.
* Bad arguments are rejected with GNP_ERR_INVALID_ARG.
"""
import numpy as np
import pytest

from oracle import krylov_ref as K
from oracle import precond_ref as PR
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


def matrices():
    return {"convdiff": I.convdiff2d(40, 100.0), "powerlaw": I.powerlaw(5000, seed=2),
            "aniso": I.aniso3d(10, 100.0)}


@pytest.mark.parametrize("kind", ["convdiff", "powerlaw", "aniso"])
def test_apply_matches_oracle(gnp, kind):
    import torch
    A = matrices()[kind]
    Mt = gnp.mat_from_csr(A)
    v = I.gaussian(A.n, seed=7)
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    Pj = gnp.gnp_precond_create(Mt, gnp.PRECOND_JACOBI)
    gnp.gnp_precond_apply(Pj, dev(v), z)
    assert np.array_equal(z.cpu().numpy(), PR.jacobi(A.to_scipy())(v))
    for iters, rtol in ((10, 1e-6), (4, 0.0), (30, 1e-3)):
        Pg = gnp.gnp_precond_create(Mt, gnp.PRECOND_GMRES, inner_iters=iters, inner_rtol=rtol)
        gnp.gnp_precond_apply(Pg, dev(v), z)
        zr, k, _ = PR.inner_gmres_solve(A.to_scipy(), v, iters, rtol)
        np.testing.assert_allclose(z.cpu().numpy(), zr, rtol=0, atol=1e-10 * np.abs(zr).max())
    # zero vector -> zero
    gnp.gnp_precond_apply(Pg, dev(np.zeros(A.n)), z)
    assert torch.count_nonzero(z).item() == 0


@pytest.mark.parametrize("kind", ["convdiff", "powerlaw"])
@pytest.mark.parametrize("prec", ["jacobi", "gmres"])
def test_fgmres_with_baseline_preconditioners_matches_oracle(gnp, kind, prec):
    import torch
    A = matrices()[kind]
    As = A.to_scipy()
    Mt = gnp.mat_from_csr(A)
    b = I.spmv(A, np.ones(A.n))  # the paper's test problem x = 1
    if prec == "jacobi":
        P = gnp.gnp_precond_create(Mt, gnp.PRECOND_JACOBI)
        op = PR.jacobi(As)
    else:
        P = gnp.gnp_precond_create(Mt, gnp.PRECOND_GMRES, inner_iters=10, inner_rtol=1e-6)
        op = PR.inner_gmres(As, 10, 1e-6)
    m, maxit = 10, 60
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = gnp.fgmres_solve(Mt, dev(b), x, P, restart=m, rtol=1e-8, maxiters=maxit)
    xr, ir = K.fgmres(As, b, op, m=m, rtol=1e-8, maxiters=maxit)
    assert info.status == ir["status"]
    assert info.iters == ir["iters"]
    h, hr = np.asarray(info.history), np.asarray(ir["history"])
    if prec == "jacobi":
        # a linear preconditioner: the two float64 runs agree to rounding
        np.testing.assert_allclose(h, hr, rtol=1e-9, atol=1e-13)
        np.testing.assert_allclose(x.cpu().numpy(), xr, rtol=0, atol=1e-7 * np.abs(xr).max())
    else:
        # inner GMRES is nonlinear, and on the row-scaled power-law matrix its least-squares
        # solutions amplify rounding: bound the GPU-oracle gap by the oracle's own spread
        # under float64-rounding-sized perturbations of every input vector
        rng = np.random.default_rng(0)
        spread = np.zeros_like(hr)
        for _ in range(3):
            opp = lambda v: op(v * (1.0 + 2.2e-16 * rng.standard_normal(v.shape)))
            _, ip = K.fgmres(As, b, opp, m=m, rtol=1e-8, maxiters=maxit)
            hp = np.asarray(ip["history"])
            k = min(len(hp), len(hr))
            spread[:k] = np.maximum(spread[:k], np.abs(hp[:k] - hr[:k]) / hr[:k])
            spread[k:] = np.maximum(spread[k:], spread[:k].max())
        np.testing.assert_allclose(h[:6], hr[:6], rtol=1e-9, atol=1e-13)
        dev_rel = np.abs(h - hr) / hr
        assert np.all(dev_rel <= 10.0 * spread + 1e-9), (dev_rel.max(), spread.max())


def test_handle_identity_and_gnp_equal_the_direct_calls(gnp):
    import torch
    A = I.convdiff2d(32, 100.0)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=4), I.init_weights(4, seed=3))
    b = dev(I.spmv(A, np.ones(A.n)))
    for kind, model in ((gnp.PRECOND_IDENTITY, None), (gnp.PRECOND_GNP, M)):
        P = gnp.gnp_precond_create(Mt, kind, M=model)
        x1 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        x2 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        i1 = gnp.fgmres_solve(Mt, b, x1, model, restart=20, rtol=1e-8, maxiters=200)
        i2 = gnp.fgmres_solve(Mt, b, x2, P, restart=20, rtol=1e-8, maxiters=200)
        assert i1.status == i2.status and i1.iters == i2.iters
        assert np.array_equal(i1.history, i2.history) and torch.equal(x1, x2)
    # gnp_precond_apply of the GNP kind widens gnp_apply's float32 output
    P = gnp.gnp_precond_create(Mt, gnp.PRECOND_GNP, M=M)
    v = dev(I.gaussian(A.n, seed=1))
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    zf = torch.empty(A.n, dtype=torch.float32, device="cuda")
    gnp.gnp_precond_apply(P, v, z)
    gnp.gnp_apply(M, v, zf)
    assert torch.equal(z, zf.double())


def test_bad_arguments(gnp):
    A = I.poisson2d(8)
    B = I.poisson2d(9)
    Mt, Mb = gnp.mat_from_csr(A), gnp.mat_from_csr(B)
    M = gnp.gnp_create(Mt, gnp.make_config(L=1), I.init_weights(1, seed=0))
    for kw in (dict(kind=gnp.PRECOND_GMRES, inner_iters=0), dict(kind=gnp.PRECOND_GMRES, inner_iters=129),
               dict(kind=gnp.PRECOND_GNP), dict(kind=7)):
        with pytest.raises(gnp.GnpError) as ei:
            gnp.gnp_precond_create(Mt, **kw)
        assert ei.value.status == 1
    with pytest.raises(gnp.GnpError):
        gnp.gnp_precond_create(Mb, gnp.PRECOND_GNP, M=M)
