"""Philox4x32-10 and Box-Muller, written from their published definitions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Philox4x32 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11): a 4 x 32-bit counter and a 2 x 32-bit key; each of the 10 rounds replaces
(c0, c1, c2, c3) by (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the Weyl
constants (0x9E3779B9, 0xBB67AE85).

Draw convention used by the training sampler (the CUDA side implements the same
convention independently):
* key = (seed mod 2^32, seed div 2^32);
* counter = (idx mod 2^32, idx div 2^32, step, stream), one call per group of four
  consecutive elements (idx = element // 4);
* uniform U(r) = ((r >> 9) + 0.5) * 2^-23 = (2 (r >> 9) + 1) * 2^-24: at most 24
  significant bits, so exactly representable in float32, and inside (0, 1);
* Box-Muller per word pair (r0, r1) and (r2, r3):
  rho = sqrt(-2 ln U(r_even)), theta = 2 pi U(r_odd); outputs rho cos theta, rho sin theta.
Element e of a stream is output (e mod 4) of call e // 4, in the order
[rho01 cos, rho01 sin, rho23 cos, rho23 sin].

Streams: 1 = Gaussian solutions x of a training batch, 2 = the epsilon of Eq. 5,
3 = the Arnoldi start vector of the sampler.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)

STREAM_X = 1
STREAM_EPS = 2
STREAM_V1 = 3


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """ctr: uint32-valued array [..., 4]; key: (k0, k1).  Returns uint32 [..., 4]."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0, k1 = key[0] & 0xFFFFFFFF, key[1] & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack(c, axis=-1).astype(np.uint32)


def uniform24(r: np.ndarray) -> np.ndarray:
    return ((r.astype(np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def raw_words(count: int, seed: int, step: int, stream: int) -> np.ndarray:
    """The uint32 words of calls idx = 0 .. ceil(count/4)-1, shape [calls, 4]."""
    calls = (count + 3) // 4
    idx = np.arange(calls, dtype=np.uint64)
    ctr = np.zeros((calls, 4), dtype=np.uint64)
    ctr[:, 0] = idx & MASK
    ctr[:, 1] = idx >> np.uint64(32)
    ctr[:, 2] = step & 0xFFFFFFFF
    ctr[:, 3] = stream & 0xFFFFFFFF
    return philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))


def normal(count: int, seed: int, step: int, stream: int) -> np.ndarray:
    """``count`` N(0,1) float64 draws of (seed, step, stream) under the convention above."""
    w = raw_words(count, seed, step, stream)
    rho01 = np.sqrt(-2.0 * np.log(uniform24(w[:, 0])))
    th01 = 2.0 * np.pi * uniform24(w[:, 1])
    rho23 = np.sqrt(-2.0 * np.log(uniform24(w[:, 2])))
    th23 = 2.0 * np.pi * uniform24(w[:, 3])
    out = np.stack([rho01 * np.cos(th01), rho01 * np.sin(th01),
                    rho23 * np.cos(th23), rho23 * np.sin(th23)], axis=-1).reshape(-1)
    return out[:count]
