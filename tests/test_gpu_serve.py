"""The continuous-batching solve server (gnp_server_*) on the GPU.

* Each request's result is the same alone and in a mix of concurrently running requests
  of different sizes, families and preconditioners (and equal to a lone fgmres_solve).
* Admission by device-memory footprint: a budget for one request at a time still
  completes every request; a request larger than the whole budget fails with
  GNP_ERR_OOM; a NaN right-hand side gives GNP_ERR_NAN; a wait that runs out returns
  GNP_ERR_TIMEOUT while the request keeps running.
"""
import numpy as np
import pytest

from paper_2406_00809_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gnp():
    import torch
    from paper_2406_00809_gb300 import build, gnp as g
    build.build()
    assert torch.cuda.is_available()
    return g


def problems(g):
    """Mixed sizes and families; GNP (two share one model) and identity preconditioners."""
    import torch
    out = []
    specs = [("poisson", I.poisson2d(40), True, 0), ("convdiff", I.convdiff2d(48, 100.0), True, 1),
             ("powerlaw", I.powerlaw(6000, seed=4), True, 2), ("aniso", I.aniso3d(12, 100.0), False, 3),
             ("poisson-id", I.poisson2d(24), False, 4)]
    for name, A, use_gnp, seed in specs:
        Mt = g.mat_from_csr(A)
        M = g.gnp_create(Mt, g.make_config(L=4), I.init_weights(4, seed=seed)) if use_gnp else None
        for k in range(2 if name == "convdiff" else 1):
            b = torch.from_numpy(I.spmv(A, I.gaussian(A.n, seed=10 * seed + k))).cuda()
            out.append((name, A, Mt, M, b))
    return out


def test_alone_equals_mix_equals_direct(gnp):
    import torch
    probs = problems(gnp)
    m, rtol, maxit = 20, 1e-8, 80
    # direct solves
    direct = []
    for name, A, Mt, M, b in probs:
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        info = gnp.fgmres_solve(Mt, b, x, M, restart=m, rtol=rtol, maxiters=maxit, history=False)
        direct.append((x.clone(), info))
    srv = gnp.Server(max_bytes=8 << 30, max_active=16, restart=m)
    # alone: one request at a time
    alone = []
    for name, A, Mt, M, b in probs:
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        info = srv.wait(srv.submit(Mt, M, b, x, rtol, maxit))
        alone.append((x.clone(), info))
    # mix: all at once
    xs, tickets = [], []
    for name, A, Mt, M, b in probs:
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        xs.append(x)
        tickets.append(srv.submit(Mt, M, b, x, rtol, maxit))
    mix = [(xs[k], srv.wait(t)) for k, t in enumerate(tickets)]
    st = srv.stats()
    srv.close()
    assert st["max_active_seen"] >= 2
    for (name, *_), (xd, idr), (xa, ia), (xm, im) in zip(probs, direct, alone, mix):
        assert idr.status == ia.status == im.status, name
        assert idr.iters == ia.iters == im.iters, name
        scale = float(xd.abs().max())
        assert float((xa - xd).abs().max()) <= 1e-12 * scale, name
        assert float((xm - xa).abs().max()) <= 1e-12 * scale, name


def test_footprint_admission_oom_nan_timeout(gnp):
    import torch
    A = I.convdiff2d(40, 100.0)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=4), I.init_weights(4, seed=0))
    b = torch.from_numpy(I.spmv(A, I.gaussian(A.n, seed=0))).cuda()
    # budget for about one request: all still complete, never two at once
    fp = A.n * (31 * 8 + 30 * 4 + 8 + 128)  # basis, directions, w, hidden blocks
    one = int(1.5 * fp) + 100_000
    srv = gnp.Server(max_bytes=one, max_active=8, restart=30)
    xs = [torch.zeros(A.n, dtype=torch.float64, device="cuda") for _ in range(4)]
    ts = [srv.submit(Mt, M, b, x, 1e-8, 60) for x in xs]
    infos = [srv.wait(t) for t in ts]
    assert all(i.iters == infos[0].iters for i in infos)
    assert srv.stats()["max_active_seen"] == 1
    # larger than the whole budget
    big = I.poisson2d(300)
    Mb = gnp.mat_from_csr(big)
    bb = torch.ones(big.n, dtype=torch.float64, device="cuda")
    xb = torch.zeros(big.n, dtype=torch.float64, device="cuda")
    assert srv.wait(srv.submit(Mb, None, bb, xb, 1e-8, 50)).status == 3  # GNP_ERR_OOM
    # NaN right-hand side
    bn = b.clone()
    bn[5] = float("nan")
    xn = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    assert srv.wait(srv.submit(Mt, M, bn, xn, 1e-8, 60)).status == 10  # GNP_ERR_NAN
    srv.close()
    # a wait that runs out leaves the request running
    srv = gnp.Server(max_bytes=8 << 30, max_active=4, restart=30)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    t = srv.submit(Mt, M, b, x, 1e-30, 3000)
    with pytest.raises(gnp.GnpError) as ei:
        srv.wait(t, timeout=1e-4)
    assert ei.value.status == 9
    info = srv.wait(t, timeout=600)
    assert info.status == 8 and info.iters == 3000
    srv.close()
