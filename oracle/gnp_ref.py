"""Oracle for the GNP operator M (Sec. 2.3) and its training pieces (Sec. 2.2, Sec. 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain float64 numpy/scipy.

Shapes: a right-hand side batch ``b`` is [n, B]; hidden blocks are [n, B, d] with
d = 16; the matrix is a scipy CSR built from ``inputs.CSR``.

Readings of the paper taken here (where it is silent):
* no activation after the encoder output nor after the decoder output; biases only in
  the MLPs, none in Res-GCONV (Eq. 7 has none);
* tau = ||b||_2 = 0 gives M(0) = 0;
* the l1 training loss is averaged over the n*B entries; sign(0) = 0 and ReLU'(0) = 0;
* Adam: beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias corrected.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

D = 16
HID = 32

FORM_PAPER = 0   # Res-GCONV(X) = ReLU(X U + A_hat X W)           (Eq. 7)
FORM_RESID = 1   # X + ReLU(A_hat X W)                              (residual variant)


# ----------------------------------------------------------------------------- Eq. 6

def gamma(A: sp.csr_matrix) -> float:
    """gamma = min( max_i sum_j |a_ij| , max_j sum_i |a_ij| )   (Eq. 6)."""
    absA = abs(A)
    row_max = np.asarray(absA.sum(axis=1)).max() if A.shape[0] else 0.0
    col_max = np.asarray(absA.sum(axis=0)).max() if A.shape[1] else 0.0
    return float(min(row_max, col_max))


def normalise(A: sp.csr_matrix) -> sp.csr_matrix:
    """A_hat = A / gamma   (Eq. 6)."""
    return (A / gamma(A)).tocsr()


# ----------------------------------------------------------------------- weight blob

def unpack(blob: np.ndarray, L: int) -> dict:
    """Split the flat weight blob (order documented in include/gnp.h) into float64 arrays.

    Every matrix multiplies from the right: layer output = input @ W + b (Sec. 2.3,
    where GCONV is written ReLU(A_hat X W) with W of shape d_in x d_out).
    """
    w = np.asarray(blob, dtype=np.float64)
    p = 0

    def take(*shape):
        nonlocal p
        k = int(np.prod(shape))
        out = w[p:p + k].reshape(shape)
        p += k
        return out

    P = {}
    P["enc_W1"] = take(1, HID)
    P["enc_b1"] = take(HID)
    P["enc_W2"] = take(HID, D)
    P["enc_b2"] = take(D)
    P["U"] = []
    P["W"] = []
    for _ in range(L):
        P["U"].append(take(D, D))
        P["W"].append(take(D, D))
    P["dec_W1"] = take(D, HID)
    P["dec_b1"] = take(HID)
    P["dec_W2"] = take(HID, 1)
    P["dec_b2"] = take(1)
    assert p == w.size, (p, w.size)
    return P


def pack(P: dict) -> np.ndarray:
    parts = [P["enc_W1"], P["enc_b1"], P["enc_W2"], P["enc_b2"]]
    for U, W in zip(P["U"], P["W"]):
        parts += [U, W]
    parts += [P["dec_W1"], P["dec_b1"], P["dec_W2"], P["dec_b2"]]
    return np.concatenate([np.ravel(x) for x in parts])


def relu(x):
    return np.maximum(x, 0.0)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 the way a float32 store to a bfloat16 hidden block does: first to
    float32, then to the upper 16 bits of the float32 pattern, round to nearest, ties to
    even (add 0x7FFF plus the lowest kept bit, clear the low 16 bits).  Returned as
    float64.  Inputs are finite."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def spmm(Ahat: sp.csr_matrix, X: np.ndarray) -> np.ndarray:
    """A_hat X for X of shape [n, B, d] (the sparse product is the library primitive)."""
    n, B, d = X.shape
    return np.asarray(Ahat @ X.reshape(n, B * d)).reshape(n, B, d)


def spmm_T(Ahat: sp.csr_matrix, X: np.ndarray) -> np.ndarray:
    """A_hat^T X for X of shape [n, B, d]."""
    n, B, d = X.shape
    return np.asarray(Ahat.T @ X.reshape(n, B * d)).reshape(n, B, d)


# ------------------------------------------------------------------- forward (M(b))

def scale(b: np.ndarray):
    """s(b) = (sqrt(n)/tau) b with tau = ||b||_2 per column (Eq. 8).

    Returns (u, tau).  Columns with tau = 0 give u = 0.
    """
    n = b.shape[0]
    tau = np.sqrt((b * b).sum(axis=0))
    f = np.where(tau > 0, np.sqrt(n) / np.where(tau > 0, tau, 1.0), 0.0)
    return b * f, tau


def forward(Ahat: sp.csr_matrix, b: np.ndarray, P: dict, form: int = FORM_PAPER,
            keep: bool = False, scaled: bool = True, hstore: str = "f64"):
    """z = M(b) for b of shape [n] or [n, B] (Sec. 2.3, Fig. 1, Eqs. 6-8).

    s -> encoder (1 -> 32, ReLU, -> 16) -> L x Res-GCONV -> decoder (16 -> 32, ReLU,
    -> 1) -> s^{-1}.  With keep=True also returns the saved activations for backward.
    scaled=False is the ablation of Sec. 4 without s: the network sees b itself and its
    output is z.  hstore="bf16" emulates a bfloat16 hidden block (reading c18): every
    hidden block that is stored between two steps -- the encoder output and the output
    of each layer but the last, which the decoder consumes directly -- is rounded with
    round_bf16; all arithmetic stays float64.
    """
    if hstore not in ("f64", "bf16"):
        raise ValueError(hstore)
    store = round_bf16 if hstore == "bf16" else (lambda X: X)
    vec = b.ndim == 1
    bb = b[:, None] if vec else b
    n = bb.shape[0]
    if scaled:
        u, tau = scale(bb)
    else:
        u, tau = bb.copy(), np.full(bb.shape[1], np.sqrt(n))
    a1 = u[:, :, None] * P["enc_W1"][0][None, None, :] + P["enc_b1"]   # [n,B,32]
    r1 = relu(a1)
    H = store(r1 @ P["enc_W2"] + P["enc_b2"])                           # [n,B,16]
    Hs = [H]
    Ps, pres = [], []
    L = len(P["U"])
    for l, (U, W) in enumerate(zip(P["U"], P["W"])):
        X = Hs[-1]
        AX = spmm(Ahat, X)
        if form == FORM_PAPER:
            pre = X @ U + AX @ W
            Hn = relu(pre)
        else:
            pre = AX @ W
            Hn = X + relu(pre)
        if l < L - 1:
            Hn = store(Hn)
        Ps.append(AX)
        pres.append(pre)
        Hs.append(Hn)
    c1 = Hs[-1] @ P["dec_W1"] + P["dec_b1"]                            # [n,B,32]
    q = relu(c1)
    o = (q @ P["dec_W2"])[:, :, 0] + P["dec_b2"][0]                     # [n,B]
    back = np.where(tau > 0, tau / np.sqrt(n), 0.0)
    z = o * back
    z = z[:, 0] if vec else z
    if not keep:
        return z
    cache = dict(u=u, tau=tau, a1=a1, r1=r1, Hs=Hs, Ps=Ps, pres=pres, c1=c1, q=q,
                 back=back, form=form)
    return z, cache


def hidden_trace(Ahat, b, P, form=FORM_PAPER):
    """The hidden blocks H^0..H^L for a single right-hand side b [n] (each [n, 16])."""
    _, cache = forward(Ahat, b[:, None], P, form, keep=True)
    return [H[:, 0, :] for H in cache["Hs"]]


# ------------------------------------------------------------------------ backward

def backward(Ahat: sp.csr_matrix, P: dict, cache: dict, dz: np.ndarray) -> dict:
    """Gradients of a scalar loss w.r.t. all weights given dL/dz [n, B].

    Chain rule through s^{-1}, decoder, the L layers and the encoder; tau depends only
    on b, so it carries no gradient (App. E: backward uses the same products with A_hat
    and with tall n-row matrices as forward).
    """
    form = cache["form"]
    do = dz * cache["back"][None, :]                                   # [n,B]
    q, c1 = cache["q"], cache["c1"]
    G = {}
    G["dec_W2"] = np.einsum("nbh,nb->h", q, do)[:, None]
    G["dec_b2"] = np.array([do.sum()])
    dq = do[:, :, None] * P["dec_W2"][:, 0][None, None, :]
    dc1 = dq * (c1 > 0)
    HL = cache["Hs"][-1]
    G["dec_W1"] = np.einsum("nbi,nbj->ij", HL, dc1)
    G["dec_b1"] = dc1.sum(axis=(0, 1))
    dH = dc1 @ P["dec_W1"].T
    L = len(P["U"])
    GU = [None] * L
    GW = [None] * L
    for l in reversed(range(L)):
        X = cache["Hs"][l]
        AX = cache["Ps"][l]
        pre = cache["pres"][l]
        Gp = dH * (pre > 0)
        W = P["W"][l]
        GW[l] = np.einsum("nbi,nbj->ij", AX, Gp)
        if form == FORM_PAPER:
            U = P["U"][l]
            GU[l] = np.einsum("nbi,nbj->ij", X, Gp)
            dH = Gp @ U.T + spmm_T(Ahat, Gp @ W.T)
        else:
            GU[l] = np.zeros((D, D))
            dH = dH + spmm_T(Ahat, Gp @ W.T)
    G["U"], G["W"] = GU, GW
    r1, a1, u = cache["r1"], cache["a1"], cache["u"]
    G["enc_W2"] = np.einsum("nbh,nbj->hj", r1, dH)
    G["enc_b2"] = dH.sum(axis=(0, 1))
    dr1 = dH @ P["enc_W2"].T
    da1 = dr1 * (a1 > 0)
    G["enc_W1"] = np.einsum("nb,nbh->h", u, da1)[None, :]
    G["enc_b1"] = da1.sum(axis=(0, 1))
    return G


# ---------------------------------------------------------------------- loss (Sec. 3)

def l1_loss(Asys: sp.csr_matrix, z: np.ndarray, b: np.ndarray):
    """l = mean |A z - b| over the n*B entries (the l1 residual loss with b = A x).

    Returns (loss, dL/dz) with dL/dz = A^T sign(A z - b) / (n B).
    """
    r = np.asarray(Asys @ z) - b
    nB = r.size
    loss = np.abs(r).sum() / nB
    dz = np.asarray(Asys.T @ np.sign(r)) / nB
    return float(loss), dz


# ----------------------------------------------------------------------------- Adam

class Adam:
    """Adam (Kingma & Ba) over the flat blob: lr 1e-3 (Sec. 3), beta 0.9/0.999, eps 1e-8."""

    def __init__(self, nparam, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(nparam)
        self.v = np.zeros(nparam)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, w: np.ndarray, g: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return w - self.lr * mh / (np.sqrt(vh) + self.eps)


def train_step(Ahat, w_blob, L, form, x, opt: Adam, scaled: bool = True, b=None):
    """One training step on given solution vectors x [n, B] (b = A_hat x), or on given
    right-hand sides b [n, B] when x is None (the b ~ N(0, I) ablation of Sec. 4).

    The system used for training is the prescaled one, A <- A / gamma (Sec. 3
    "Problems"), which equals A_hat.  Returns (new blob, loss before the update).
    """
    if x is not None:
        b = np.asarray(Ahat @ x)
    P = unpack(w_blob, L)
    z, cache = forward(Ahat, b, P, form, keep=True, scaled=scaled)
    loss, dz = l1_loss(Ahat, z, b)
    G = backward(Ahat, P, cache, dz)
    g = pack(G)
    return opt.step(np.asarray(w_blob, dtype=np.float64), g), loss
