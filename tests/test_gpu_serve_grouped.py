"""The solve server's grouped steps (gnp_server_config.grouped = 1) on the GPU.

Requests whose GNP runs on the short-row layer kernels advance together, one FGMRES step
per round, every kernel of the step launched once for all of them over a work table.  Each
grouped request must compute exactly what a lone fgmres_solve computes with the two-pass
CGS2 schedule (GNP_ORTHO=cgs2), alone and in a mix: the mix below has more grouped
requests than one grouped GNP launch takes (six), both hidden precisions and both layer
forms, different depths L and sizes, a GNP with trained weights whose solve converges
inside a cycle, a 16-row system whose Krylov space is exhausted (breakdown), and requests
that run per request beside them (a power-law matrix whose long rows need the tile kernels,
and no preconditioner).
"""
import os

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
    import torch
    out = []
    specs = [  # name, matrix, L, form, hprec (None: no preconditioner), seed
        ("poisson-fp32", I.poisson2d(40), 4, g.LAYER_PAPER, g.H_FP32, 0),
        ("convdiff-fp32", I.convdiff2d(48, 100.0), 4, g.LAYER_PAPER, g.H_FP32, 1),
        ("convdiff-L2", I.convdiff2d(36, 100.0), 2, g.LAYER_PAPER, g.H_FP32, 2),
        ("aniso-fp32", I.aniso3d(12, 100.0), 3, g.LAYER_PAPER, g.H_FP32, 3),
        ("convdiff-bf16", I.convdiff2d(44, 100.0), 4, g.LAYER_PAPER, g.H_BF16, 4),
        ("poisson-bf16", I.poisson2d(52), 4, g.LAYER_PAPER, g.H_BF16, 5),
        ("convdiff-resid", I.convdiff2d(40, 100.0), 4, g.LAYER_RESID, g.H_FP32, 6),
        ("poisson-small", I.poisson2d(20), 4, g.LAYER_PAPER, g.H_FP32, 7),
        ("powerlaw", I.powerlaw(6000, seed=4), 4, g.LAYER_PAPER, g.H_FP32, 8),
        ("poisson-id", I.poisson2d(24), 0, None, None, 9),
        ("convdiff64-trained", I.convdiff2d(64, 100.0), 8, g.LAYER_PAPER, g.H_FP32, -1),
        ("poisson4-breakdown", I.poisson2d(4), 2, g.LAYER_PAPER, g.H_FP32, 11),
    ]
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gnp_convdiff64_weights.npy")
    for name, A, L, form, hprec, seed in specs:
        Mt = g.mat_from_csr(A)
        M = None
        if hprec is not None:
            w = np.load(golden) if seed < 0 else I.init_weights(L, seed=seed)
            M = g.gnp_create(Mt, g.make_config(L=L, form=form, hprec=hprec), w)
        for k in range(2 if name == "convdiff-fp32" else 1):
            b = torch.from_numpy(I.spmv(A, I.gaussian(A.n, seed=abs(10 * seed + k)))).cuda()
            out.append((name, A, Mt, M, b))
    return out


def test_grouped_alone_equals_mix_equals_direct(gnp, monkeypatch):
    import torch
    monkeypatch.setenv("GNP_ORTHO", "cgs2")  # the schedule the grouped step follows
    probs = problems(gnp)
    n_grouped = sum(1 for _, A, _, M, _ in probs if M is not None and int(np.diff(A.row_ptr).max()) <= 16)
    assert n_grouped > 6  # more than one grouped launch's worth
    m, rtol, maxit = 20, 1e-8, 100
    direct = []
    for name, A, Mt, M, b in probs:
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        info = gnp.fgmres_solve(Mt, b, x, M, restart=m, rtol=rtol, maxiters=maxit, history=False)
        direct.append((x.clone(), info))
    srv = gnp.Server(max_bytes=8 << 30, max_active=16, restart=m, grouped=True)
    alone = []
    for name, A, Mt, M, b in probs:
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        info = srv.wait(srv.submit(Mt, M, b, x, rtol, maxit))
        alone.append((x.clone(), info))
    xs, tickets = [], []
    for name, A, Mt, M, b in probs:
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        xs.append(x)
        tickets.append(srv.submit(Mt, M, b, x, rtol, maxit))
    mix = [(xs[k], srv.wait(t)) for k, t in enumerate(tickets)]
    st = srv.stats()
    srv.close()
    assert st["max_active_seen"] > 6  # the mix ran more requests at once than one grouped launch takes
    for (name, *_), (xd, idr), (xa, ia), (xm, im) in zip(probs, direct, alone, mix):
        assert idr.status == ia.status == im.status, name
        assert idr.iters == ia.iters == im.iters, name
        assert idr.cycles == ia.cycles == im.cycles, name
        scale = float(xd.abs().max())
        assert float((xa - xd).abs().max()) <= 1e-12 * scale, name
        assert float((xm - xa).abs().max()) <= 1e-12 * scale, name
    # the stopping rule ended the trained and the 16-row solves inside a cycle
    for (name, *_), (_, i) in zip(probs, mix):
        if name in ("convdiff64-trained", "poisson4-breakdown"):
            assert i.status == 0 and i.iters % m != 0, (name, i.status_name, i.iters)


def test_grouped_stream_stops_and_budget(gnp, monkeypatch):
    """A stream longer than the slots (four at a time), with solves that cannot reach their
    rtol (far below rounding) next to converging ones and different iteration caps: every
    request completes with the status, iteration count and solution of its lone solve."""
    import torch
    monkeypatch.setenv("GNP_ORTHO", "cgs2")
    A = I.convdiff2d(40, 100.0)
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=4), I.init_weights(4, seed=0))
    reqs = []
    for k in range(12):
        b = torch.from_numpy(I.spmv(A, I.gaussian(A.n, seed=100 + k))).cuda()
        rtol = 1e-30 if k % 3 == 0 else 1e-8
        reqs.append((b, rtol, 60 + 10 * (k % 4)))
    want = []
    for b, rtol, maxit in reqs:
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        info = gnp.fgmres_solve(Mt, b, x, M, restart=30, rtol=rtol, maxiters=maxit, history=False)
        want.append((x, info))
    srv = gnp.Server(max_bytes=8 << 30, max_active=4, restart=30, grouped=True)
    xs = [torch.zeros(A.n, dtype=torch.float64, device="cuda") for _ in reqs]
    ts = [srv.submit(Mt, M, b, x, rtol, maxit) for x, (b, rtol, maxit) in zip(xs, reqs)]
    got = [srv.wait(t) for t in ts]
    st = srv.stats()
    srv.close()
    assert 2 <= st["max_active_seen"] <= 4
    for (xw, iw), x, i in zip(want, xs, got):
        assert i.status == iw.status and i.iters == iw.iters
        assert float((x - xw).abs().max()) <= 1e-12 * float(xw.abs().max())
