"""GPU parity of the training path (Sec. 2.2, Sec. 3) against the float64 oracle.

* Philox4x32-10 on the device: bit-exact on the published known-answer vectors and
  on the counters the sampler uses.
* The Eq. 5 sampler: Gaussian half within float32 Box-Muller rounding; the Arnoldi half
  through Q Q^T = (H_bar^T H_bar)^-1 (independent of the SVD basis) and elementwise.
* Batched forward 1e-5, hand-written backward 1e-4 relative L2 against the oracle
  gradient; central differences on the device; the torch.autograd.Function wrapper.
* One training step: loss and the Adam update against the oracle.
"""
import os

import numpy as np
import pytest

from oracle import gnp_ref as G
from oracle import krylov_ref as K
from oracle import philox_ref as PH
from paper_2406_00809_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


@pytest.fixture(scope="module")
def gnp():
    import torch
    from paper_2406_00809_gb300 import build, gnp as g
    build.build()
    assert torch.cuda.is_available()
    return g


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


def to_i32(a):
    return np.asarray(a, dtype=np.uint64).astype(np.uint32).view(np.int32)


def test_philox_known_answers_on_device(gnp):
    import torch
    rows = [[int(t, 16) for t in l.split()] for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for r in rows:
        ctr = torch.from_numpy(to_i32([r[0:4]])).cuda()
        out = torch.empty_like(ctr)
        gnp.gnp_philox4x32_10(ctr, r[4], r[5], out)
        got = out.cpu().numpy().view(np.uint32)[0].tolist()
        assert got == r[6:10]


def test_philox_bit_exact_sampler_counters(gnp):
    import torch
    calls = 4099
    idx = np.arange(calls, dtype=np.uint64)
    ctr = np.zeros((calls, 4), dtype=np.uint64)
    ctr[:, 0] = idx & 0xFFFFFFFF
    ctr[:, 1] = idx >> np.uint64(32)
    ctr[:, 2] = 17
    ctr[:, 3] = PH.STREAM_X
    seed = 0x123456789ABCDEF
    ref = PH.philox4x32_10(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    c = torch.from_numpy(to_i32(ctr)).cuda()
    out = torch.empty_like(c)
    gnp.gnp_philox4x32_10(c, seed & 0xFFFFFFFF, seed >> 32, out)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref)


def _model(gnp, A, L, B=16, mA=12, seed=5, form=0, blob_seed=1):
    blob = I.init_weights(L, seed=blob_seed)
    blob[32:64] = np.random.default_rng(blob_seed).standard_normal(32) * 0.2
    Mt = gnp.mat_from_csr(A)
    M = gnp.gnp_create(Mt, gnp.make_config(L=L, form=form, batch=B, arnoldi_m=mA, seed=seed), blob)
    return Mt, M, blob


def test_sampler_matches_oracle(gnp):
    import torch
    A = I.convdiff2d(20, 100.0)
    n, B, mA, seed, step = A.n, 16, 10, 77, 3
    Mt, M, _ = _model(gnp, A, 2, B=B, mA=mA, seed=seed)
    x = torch.empty(n * B, dtype=torch.float32, device="cuda")
    gnp.gnp_sample_batch(M, step, x)
    xg = x.cpu().numpy().reshape(n, B).astype(np.float64)
    # Gaussian half: stream 1, element (i, c) -> index i*Bg + c
    Ba = B // 2
    gref = PH.normal(n * (B - Ba), seed, step, PH.STREAM_X).reshape(n, B - Ba)
    np.testing.assert_allclose(xg[:, Ba:], gref, rtol=0, atol=2e-5 * np.abs(gref).max())
    # Arnoldi half: x = V_m Q eps on A_hat from the seed's start vector
    Ahat = G.normalise(A.to_scipy())
    V, H = K.arnoldi(Ahat, K.arnoldi_v1(n, seed), mA)
    Q, s = K.sampler_matrix(H)
    xr = K.training_x(V, Q, Ba, B - Ba, seed, step)
    assert rel(xg[:, :Ba], xr[:, :Ba]) <= 1e-4
    # covariance pin independent of the singular-vector basis: x in range(V_m)
    Vm = V[:, :mA]
    res = xg[:, :Ba] - Vm @ (Vm.T @ xg[:, :Ba])
    assert np.linalg.norm(res) <= 1e-4 * np.linalg.norm(xg[:, :Ba])


def _batch(n, B, seed):
    return np.random.default_rng(seed).standard_normal((n, B))


@pytest.mark.parametrize("bwd", ["tc", "row2", "quad"])
@pytest.mark.parametrize("form", [0, 1])
def test_forward_backward_batch_match_oracle(gnp, form, bwd, monkeypatch):
    """The batched forward and the hand-written backward against the float64 oracle; the
    layer backward in each of its forms (tensor cores with three TF32 products, float32
    with two rows per thread, float32 with four threads per row)."""
    import torch
    monkeypatch.setenv("GNP_TRAIN_BWD", bwd)
    A = I.convdiff2d(24, 100.0)
    n, B, L = A.n, 16, 3
    Mt, M, blob = _model(gnp, A, L, B=B, form=form)
    b = _batch(n, B, 1)
    c = _batch(n, B, 2)
    z = torch.empty(n * B, dtype=torch.float32, device="cuda")
    bd = torch.from_numpy(b.astype(np.float32)).cuda()
    gnp.gnp_forward_batch(M, bd, z)
    Ahat = G.normalise(A.to_scipy())
    P = G.unpack(blob, L)
    zr, cache = G.forward(Ahat, b.astype(np.float32).astype(np.float64), P, form, keep=True)
    assert rel(z.cpu().numpy().reshape(n, B), zr) <= 1e-5
    g = torch.empty(gnp.weight_count(L), dtype=torch.float32, device="cuda")
    gnp.gnp_backward_batch(M, torch.from_numpy(c.astype(np.float32)).cuda().reshape(-1), g)
    gr = G.pack(G.backward(Ahat, P, cache, c.astype(np.float32).astype(np.float64)))
    assert rel(g.cpu().numpy(), gr) <= 1e-4, rel(g.cpu().numpy(), gr)


@pytest.mark.parametrize("kind", ["poisson12", "aniso8"])
def test_backward_central_differences_on_device(gnp, kind):
    import torch
    A = I.poisson2d(12) if kind == "poisson12" else I.aniso3d(8, 100.0)
    n, B, L = A.n, 8, 2
    Mt, M, blob = _model(gnp, A, L, B=B)
    b = torch.from_numpy(_batch(n, B, 3).astype(np.float32)).cuda()
    c = torch.from_numpy(_batch(n, B, 4).astype(np.float32)).cuda()
    z = torch.empty(n * B, dtype=torch.float32, device="cuda")
    w = torch.from_numpy(blob.copy()).cuda()

    def f(wv):
        gnp.gnp_set_weights_device(M, wv)
        gnp.gnp_forward_batch(M, b, z)
        return float((z.double() * c.reshape(-1).double()).sum())

    f(w)
    g = torch.empty_like(w)
    gnp.gnp_backward_batch(M, c.reshape(-1).contiguous(), g)
    g = g.cpu().numpy()
    rng = np.random.default_rng(0)
    idx = rng.choice(w.numel(), 40, replace=False)
    h = 2e-3
    fd = []
    for k in idx:
        wp = w.clone(); wp[k] += h
        wm = w.clone(); wm[k] -= h
        fd.append((f(wp) - f(wm)) / (2 * h))
    fd = np.array(fd)
    # float32 forward, a step that rarely crosses a ReLU kink: a few percent
    assert rel(g[idx], fd) <= 5e-2, rel(g[idx], fd)


def test_autograd_function_matches_backward(gnp):
    import torch
    A = I.poisson2d(10)
    n, B, L = A.n, 8, 2
    Mt, M, blob = _model(gnp, A, L, B=B)
    Fn = gnp.gnp_function(M)
    w = torch.from_numpy(blob.copy()).cuda().requires_grad_(True)
    b = torch.from_numpy(_batch(n, B, 5).astype(np.float32)).cuda()
    z = Fn.apply(w, b)
    c = torch.from_numpy(_batch(n, B, 6).astype(np.float32)).cuda()
    (z * c).sum().backward()
    Ahat = G.normalise(A.to_scipy())
    P = G.unpack(blob, L)
    _, cache = G.forward(Ahat, b.cpu().numpy().astype(np.float64), P, 0, keep=True)
    gr = G.pack(G.backward(Ahat, P, cache, c.cpu().numpy().reshape(n, B).astype(np.float64)))
    assert rel(w.grad.cpu().numpy(), gr) <= 1e-4


def test_train_step_matches_oracle(gnp):
    import torch
    A = I.convdiff2d(16, 100.0)
    n, B, L = A.n, 8, 2
    Mt, M, blob = _model(gnp, A, L, B=B)
    x = _batch(n, B, 7).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    loss = gnp.gnp_train_step_pairs(M, xd)
    Ahat = G.normalise(A.to_scipy())
    opt = G.Adam(blob.size)
    bref = np.asarray(Ahat @ x.astype(np.float64))
    P = G.unpack(blob, L)
    z, cache = G.forward(Ahat, bref, P, 0, keep=True)
    lref, dz = G.l1_loss(Ahat, z, bref)
    assert abs(loss - lref) <= 1e-5 * lref
    g = G.pack(G.backward(Ahat, P, cache, dz))
    w1 = opt.step(blob.astype(np.float64), g)
    # the best-loss snapshot holds the weights the first loss was measured at
    np.testing.assert_array_equal(gnp.gnp_get_weights(M), blob)
    # a second step on the same pairs measures the loss at the Adam-updated weights
    loss2 = gnp.gnp_train_step_pairs(M, xd)
    z2 = G.forward(Ahat, bref, G.unpack(w1, L), 0)
    l2ref, _ = G.l1_loss(Ahat, z2, bref)
    assert abs(loss2 - l2ref) <= 2e-4 * l2ref, (loss2, l2ref)
    assert loss2 < loss


def test_training_reduces_loss_and_iterations(gnp):
    """A short training run on the Eq. 5 / Gaussian mix lowers the loss, and the trained
    GNP preconditions FGMRES better than the untrained one (Sec. 3 set-up, fewer steps)."""
    import torch
    A = I.convdiff2d(32, 100.0)
    n, L = A.n, 8
    Mt = gnp.mat_from_csr(A)
    blob = I.init_weights(L, seed=0)
    M = gnp.gnp_create(Mt, gnp.make_config(L=L, batch=16, arnoldi_m=40, seed=0), blob)
    b = torch.from_numpy(I.spmv(A, I.gaussian(n, seed=0))).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    before = gnp.fgmres_solve(Mt, b, x, M, restart=30, rtol=1e-8, maxiters=300)
    l0 = gnp.gnp_train_step(M)
    best = gnp.gnp_train(M, 400)
    assert best < 0.7 * l0, (l0, best)
    x.zero_()
    after = gnp.fgmres_solve(Mt, b, x, M, restart=30, rtol=1e-8, maxiters=300)
    assert after.status == 0, after.status_name
    assert after.iters < before.iters
    # with the trained weights the oracle takes the same number of iterations (+-2)
    w = gnp.gnp_get_weights(M)
    Ahat = G.normalise(A.to_scipy())
    P = G.unpack(w, L)
    _, ir = K.fgmres(A.to_scipy(), b.cpu().numpy(), lambda v: G.forward(Ahat, v, P, 0), m=30,
                     rtol=1e-8, maxiters=300)
    assert ir["status"] == 0
    assert abs(after.iters - ir["iters"]) <= 2, (after.iters, ir["iters"])
