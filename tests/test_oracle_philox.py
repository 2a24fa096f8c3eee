"""Pins for the oracle's Philox4x32-10 and Box-Muller (oracle/philox_ref.py)."""
import os

import numpy as np

from oracle import philox_ref as PH

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def load_kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(t, 16) for t in line.split()])
    return rows


def test_known_answer_vectors():
    rows = load_kat()
    assert len(rows) == 3
    for r in rows:
        ctr = np.array([r[0:4]], dtype=np.uint64)
        out = PH.philox4x32_10(ctr, (r[4], r[5]))[0]
        assert [int(v) for v in out] == r[6:10]


def test_uniform_is_exact_float32_open_interval():
    r = np.array([0, 0x1FF, 0x200, 0xFFFFFFFF], dtype=np.uint32)
    u = PH.uniform24(r)
    np.testing.assert_array_equal(u, [2**-24, 2**-24, 3 * 2**-24, 1 - 2**-24])
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_box_muller_first_call_by_hand():
    w = PH.raw_words(4, seed=42, step=0, stream=1)[0]
    u = [(2 * (int(t) >> 9) + 1) / 2**24 for t in w]
    rho01 = np.sqrt(-2 * np.log(u[0]))
    rho23 = np.sqrt(-2 * np.log(u[2]))
    expect = [rho01 * np.cos(2 * np.pi * u[1]), rho01 * np.sin(2 * np.pi * u[1]),
              rho23 * np.cos(2 * np.pi * u[3]), rho23 * np.sin(2 * np.pi * u[3])]
    np.testing.assert_allclose(PH.normal(4, 42, 0, 1), expect, rtol=1e-15)


def test_normal_moments_and_independence_of_streams():
    z = PH.normal(400_000, seed=1, step=3, stream=1)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1) < 0.01
    assert abs((z**4).mean() - 3) < 0.05
    z2 = PH.normal(400_000, seed=1, step=3, stream=2)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.01
    # counter layout: element 4c+k comes from call c; a prefix is stable
    np.testing.assert_array_equal(PH.normal(10, 1, 3, 1), z[:10])
