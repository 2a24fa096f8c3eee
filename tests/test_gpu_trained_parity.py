"""GNP-preconditioned FGMRES (Algorithm 1) with trained weights, GPU against the float64
oracle, at the 256 x 256 convection-diffusion size (n = 65,536, FGMRES(30), rtol 1e-8).

The weights come from the oracle alone (tests/golden/make_gnp_weights.py: 2,000 Adam
steps on the 64 x 64 problem).  With them the oracle's own iteration count moves when its
z = M(v) changes at float32 level (rounded to float32, or multiplied by 1 + 1e-7 N(0, 1)),
so the GPU's count -- float32 arithmetic, or a bfloat16 hidden block -- must lie within
that spread, +-2: tests/golden/make_iteration_bands.py records it from the oracle.  Both
hidden-block precisions, under both orthogonalisation schedules of the step (CGS2, and
the one-reduction form), must reach rtol 1e-8 in the true residual.
"""
import json
import os

import numpy as np
import pytest

from paper_2406_00809_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_weights():
    return np.load(os.path.join(GOLDEN, "gnp_convdiff64_weights.npy"))


def golden_bands():
    return json.load(open(os.path.join(GOLDEN, "gnp_iteration_bands.json")))


@pytest.fixture(scope="module")
def gnp():
    import torch
    from paper_2406_00809_gb300 import build, gnp as g
    build.build()
    assert torch.cuda.is_available()
    return g


def band(record):
    rec = golden_bands()[record]
    its = [v["iters"] for v in rec.values()]
    assert all(v["status"] == 0 for v in rec.values()), rec
    return min(its), max(its)


@pytest.mark.parametrize("ortho", ["cgs2", "dcgs2"])
@pytest.mark.parametrize("hprec", [0, 1])
def test_iterations_within_oracle_band_at_65536_rows(gnp, hprec, ortho, monkeypatch):
    import torch
    monkeypatch.setenv("GNP_ORTHO", ortho)
    A = I.convdiff2d(256, 100.0)
    b = I.spmv(A, I.gaussian(A.n, seed=0))
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=8, hprec=hprec), golden_weights())
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = gnp.fgmres_solve(Mt, torch.from_numpy(b).cuda(), x, M, restart=30, rtol=1e-8, maxiters=3000)
    lo, hi = band("convdiff256_bf16" if hprec else "convdiff256_fp32")
    assert info.status == 0, info.status_name
    assert lo - 2 <= info.iters <= hi + 2, (info.iters, lo, hi)
    r = b - A.to_scipy() @ x.cpu().numpy()
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - info.rel_res_true) <= 1e-12
