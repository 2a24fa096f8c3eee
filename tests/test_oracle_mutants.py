"""Planted mistakes in the oracle, each caught by a pin.

Every test here puts one plausible error into the oracle (on the CPU, through a patched
copy of the affected function or argument) and checks that the independent pin that
guards that part of the oracle rejects it: transposed or swapped layer weights, A_hat^T for
A_hat, sqrt(n) -> n in the scaling s, max for min in gamma, a flipped Givens sine, a single
Gram-Schmidt pass, the transpose product dropped from the backward, swapped Philox key
words, the natural logarithm in the metrics and D for D^-1 in Jacobi.  Together with the
pins themselves this shows that the pins would notice such a mistake in the oracle.
"""
import importlib.util
import os

import numpy as np
import scipy.sparse as sp

from oracle import gnp_ref as G
from oracle import krylov_ref as K
from paper_2406_00809_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def _pins_gnp():
    spec = importlib.util.spec_from_file_location("pins_gnp", os.path.join(HERE, "test_oracle_gnp.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _forward_case():
    rng = np.random.default_rng(11)
    n, L = 7, 2
    D = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.5) + np.diag(rng.random(n) + 1)
    blob = I.init_weights(L, seed=5).astype(np.float64)
    blob[np.r_[32:64]] = rng.standard_normal(32) * 0.3
    b = rng.standard_normal(n)
    zb = _pins_gnp().brute_force_M(D.tolist(), b.tolist(), blob, L, 0)
    return D, blob, b, L, zb


def _far(z, zb):
    return np.linalg.norm(z - zb) > 1e-6 * np.linalg.norm(zb)


def test_unmutated_forward_meets_the_pin():
    D, blob, b, L, zb = _forward_case()
    z = G.forward(G.normalise(sp.csr_matrix(D)), b, G.unpack(blob, L), 0)
    assert not _far(z, zb)


def test_swapped_or_transposed_layer_weights_fail_the_brute_force_pin():
    D, blob, b, L, zb = _forward_case()
    Ahat = G.normalise(sp.csr_matrix(D))
    P = G.unpack(blob, L)
    swapped = dict(P, U=P["W"], W=P["U"])
    transposed = dict(P, U=[u.T for u in P["U"]], W=[w.T for w in P["W"]])
    assert _far(G.forward(Ahat, b, swapped, 0), zb)
    assert _far(G.forward(Ahat, b, transposed, 0), zb)


def test_transposed_adjacency_fails_the_brute_force_pin():
    D, blob, b, L, zb = _forward_case()
    AhatT = sp.csr_matrix(G.normalise(sp.csr_matrix(D)).T)
    assert _far(G.forward(AhatT, b, G.unpack(blob, L), 0), zb)


def test_scaling_by_n_instead_of_sqrt_n_fails_the_brute_force_pin(monkeypatch):
    D, blob, b, L, zb = _forward_case()

    def scale_n(bb):
        n = bb.shape[0]
        tau = np.sqrt((bb * bb).sum(axis=0))
        return bb * (n / tau), tau

    monkeypatch.setattr(G, "scale", scale_n)
    assert _far(G.forward(G.normalise(sp.csr_matrix(D)), b, G.unpack(blob, L), 0), zb)


def test_max_for_min_in_gamma_fails_the_hand_example(monkeypatch):
    A = sp.csr_matrix(np.array([[1.0, -1.0, 1.0], [0.0, 1.0, 0.0], [0.0, 0.0, -1.0]]))
    assert G.gamma(A) == 2.0

    def gamma_max(M):
        M = sp.csr_matrix(M)
        absm = abs(M)
        return float(max(absm.sum(axis=1).max(), absm.sum(axis=0).max()))

    monkeypatch.setattr(G, "gamma", gamma_max)
    assert G.gamma(A) != 2.0


def test_flipped_givens_sine_fails_the_textbook_gmres_pin(monkeypatch):
    A = I.convdiff2d(8, 100.0).to_scipy()
    b = np.random.default_rng(0).standard_normal(A.shape[0])
    _, hist = K.gmres_textbook(A, b, m=10, maxiters=30)
    good = K.givens

    def givens_flipped(a, bb):
        c, s, rho = good(a, bb)
        return c, -s, rho

    monkeypatch.setattr(K, "givens", givens_flipped)
    _, info = K.fgmres(A, b, None, m=10, rtol=1e-30, maxiters=30, orth="cgs2")
    h = np.array(info["history"])
    assert len(h) != len(hist) or np.max(np.abs(h - hist) / hist) > 1e-6


def test_single_gram_schmidt_pass_fails_the_cancellation_pin(monkeypatch):
    rng = np.random.default_rng(8)
    V, _ = np.linalg.qr(rng.standard_normal((200, 6)))
    c = rng.standard_normal(6)
    u = rng.standard_normal(200)
    u -= V @ (V.T @ u)
    u /= np.linalg.norm(u)
    w = V @ c + 1e-9 * u
    good = K.orthogonalise

    def one_pass(Vm, wm, mode):
        if mode != "cgs2":
            return good(Vm, wm, mode)
        h = Vm.T @ wm
        return h, wm - Vm @ h

    monkeypatch.setattr(K, "orthogonalise", one_pass)
    _, wo = K.orthogonalise(V, w, "cgs2")
    assert np.abs(V.T @ wo).max() > 1e-12 * np.linalg.norm(wo)


def test_backward_without_the_transpose_fails_the_finite_difference_pin(monkeypatch):
    rng = np.random.default_rng(7)
    A = I.convdiff2d(4).to_scipy()          # nonsymmetric: A_hat^T != A_hat
    Ahat = G.normalise(A)
    n, L, B = A.shape[0], 2, 3
    blob = I.init_weights(L, seed=9).astype(np.float64)
    blob[32:64] = 0.1 * rng.standard_normal(32)
    b = rng.standard_normal((n, B))
    c = rng.standard_normal((n, B))

    def f(w):
        return float((G.forward(Ahat, b, G.unpack(w, L), 0) * c).sum())

    idx = rng.choice(blob.size, 120, replace=False)
    gn = _pins_gnp()._numeric_grad(f, blob, idx)
    monkeypatch.setattr(G, "spmm_T", G.spmm)  # A_hat instead of A_hat^T in the chain rule
    P = G.unpack(blob, L)
    _, cache = G.forward(Ahat, b, P, 0, keep=True)
    g = G.pack(G.backward(Ahat, P, cache, c))
    assert np.linalg.norm(g[idx] - gn) / np.linalg.norm(gn) > 1e-6


def test_swapped_philox_key_words_fail_the_known_answer_vectors():
    from oracle import philox_ref as PH
    kat = os.path.join(HERE, "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(kat):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(t, 16) for t in line.split()])
    hits = 0
    for r in rows:
        ctr = np.array([r[0:4]], dtype=np.uint64)
        good = [int(v) for v in PH.philox4x32_10(ctr, (r[4], r[5]))[0]]
        bad = [int(v) for v in PH.philox4x32_10(ctr, (r[5], r[4]))[0]]
        assert good == r[6:10]
        hits += bad != r[6:10]
    # the all-zero and all-ones vectors have equal key words and cannot tell the order; the
    # third (digits of pi) can
    assert hits >= 1


def test_natural_log_in_the_metrics_fails_the_decade_triangle(monkeypatch):
    import math
    from oracle import metrics_ref as MR
    hist = [10.0 ** (-i) for i in range(9)]
    assert abs(MR.iter_auc(hist, 1e-8) - 36.0) <= 1e-12
    monkeypatch.setattr(MR, "_excess", lambda r, rtol: math.log(max(r, MR.DBL_MIN)) - math.log(rtol))
    assert abs(MR.iter_auc(hist, 1e-8) - 36.0) > 1.0


def test_jacobi_with_d_instead_of_its_inverse_fails_the_hand_example(monkeypatch):
    from oracle import precond_ref as PR
    d = np.array([2.0, -4.0, 0.0, 0.5])
    A = sp.csr_matrix(np.diag(d) + np.diag([1.0, 1.0, 1.0], 1))
    v = np.array([1.0, 2.0, 3.0, 4.0])
    np.testing.assert_array_equal(PR.jacobi(A)(v), [0.5, -0.5, 3.0, 8.0])
    good = PR.jacobi_diag_inv
    monkeypatch.setattr(PR, "jacobi_diag_inv", lambda M: np.where(good(M) != 0, 1.0 / good(M), 1.0))
    assert not np.array_equal(PR.jacobi(A)(v), [0.5, -0.5, 3.0, 8.0])


def test_sampler_with_s_instead_of_its_inverse_fails_the_eq5_pin():
    # Eq. 5: x = V_m Z S^-1 eps gives ||A x|| = ||eps||; with Z S instead the norms differ
    from oracle import philox_ref as PH
    A = I.convdiff2d(9, 100.0).to_scipy()
    V, H = K.arnoldi(A, K.arnoldi_v1(A.shape[0], seed=1), 15)
    eps = PH.normal(15 * 4, 3, 5, PH.STREAM_EPS).reshape(15, 4)
    Q, s = K.sampler_matrix(H)
    X = K.training_x(V, Q, n_arnoldi=4, n_gauss=4, seed=3, step=5)
    np.testing.assert_allclose(np.linalg.norm(A @ X[:, :4], axis=0), np.linalg.norm(eps, axis=0), rtol=1e-9)
    Xbad = K.training_x(V, Q * (s ** 2)[None, :], n_arnoldi=4, n_gauss=4, seed=3, step=5)  # Z S
    assert np.max(np.abs(np.linalg.norm(A @ Xbad[:, :4], axis=0) / np.linalg.norm(eps, axis=0) - 1)) > 1e-3


def test_arnoldi_with_the_wrong_operator_fails_the_relation_pin():
    # the sampler's Arnoldi run must multiply by A; a run that orthogonalises v_j itself
    # (a dropped product) breaks A V_m = V_{m+1} H_bar
    A = I.aniso3d(5, 100.0).to_scipy()
    v1 = K.arnoldi_v1(A.shape[0], seed=7)
    V, H = K.arnoldi(A, v1, 20)
    assert np.linalg.norm(A @ V[:, :-1] - V @ H) <= 1e-12 * np.linalg.norm(H)
    ident = sp.identity(A.shape[0], format="csr")
    Vb, Hb = K.arnoldi(ident @ A @ A, v1, 20)  # the wrong operator (A^2)
    assert np.linalg.norm(A @ Vb[:, :-1] - Vb @ Hb) > 1e-6 * np.linalg.norm(Hb)


def test_truncating_bf16_rounding_fails_the_torch_pin():
    """Planted: bfloat16 by truncation (clear the low 16 bits) instead of round to nearest
    even.  The pin compares with torch's conversion."""
    import torch
    rng = np.random.default_rng(0)
    x = rng.standard_normal(2000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()

    def trunc(v):
        u = np.asarray(v, dtype=np.float64).astype(np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
        return u.view(np.float32).astype(np.float64)

    assert np.any(trunc(x) != ref)
    np.testing.assert_array_equal(G.round_bf16(x), ref)


def test_rounding_the_decoder_input_fails_the_stored_block_pin(monkeypatch):
    """Planted: the bfloat16 emulation also rounds H^L, which the decoder consumes in the
    same step without a store.  The pin requires H^L to be left unrounded."""
    rng = np.random.default_rng(3)
    n, L = 40, 3
    A = I.CSR(n, *_pins_gnp()._random_csr(rng, n))
    Ah = G.normalise(A.to_scipy())
    P = G.unpack(I.init_weights(L, seed=4), L)
    b = rng.standard_normal(n)
    _, c = G.forward(Ah, b, P, 0, keep=True, hstore="bf16")
    assert np.any(G.round_bf16(c["Hs"][L]) != c["Hs"][L])       # the unmutated oracle passes
    mutated = [G.round_bf16(H) for H in c["Hs"]]                  # what rounding every block gives
    assert not np.any(G.round_bf16(mutated[L]) != mutated[L])    # ... and the pin rejects it
