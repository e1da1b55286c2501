"""Pins of the oracle's random numbers and direction sampling (no GPU).

The Monte-Carlo estimator of Eq. 7 is driven by Philox4x32-10 and cosine-weighted
directions; these tests tie both to facts outside the oracle: the generator's
published known answers, uniformity, and the closed-form moments of the cosine
distribution (E[cos] = 2/3, E[cos^2] = 1/2).
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle_mod):
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle_mod.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def test_philox_uniform_and_uncorrelated(oracle_mod):
    # chi-square over 64 bins of the 24-bit uniforms of 2^14 counters x 4 words
    n = 1 << 14
    vals = np.array([oracle_mod.philox4x32_10([i, 7, 3, 1], [11, 13]) for i in range(n)], np.uint64)
    u = (vals >> 8).astype(np.float64) / 2.0 ** 24
    hist = np.bincount((u.ravel() * 64).astype(int), minlength=64)
    expect = u.size / 64
    chi2 = ((hist - expect) ** 2 / expect).sum()
    assert chi2 < 63 + 5 * np.sqrt(2 * 63)  # 5 sigma of chi^2_63
    # lag-1 serial correlation along the counter and across output words
    for a, b in [(u[:-1, 0], u[1:, 0]), (u[:, 0], u[:, 1]), (u[:, 2], u[:, 3])]:
        r = np.corrcoef(a, b)[0, 1]
        assert abs(r) < 5 / np.sqrt(a.size)


def test_sincos_turn_float_matches_libm(oracle_mod):
    m = np.concatenate([np.arange(0, 1 << 24, 61, dtype=np.uint32),
                        np.array([0, 1 << 21, 1 << 22, 3 << 21, 1 << 23, 3 << 22, (1 << 24) - 1], np.uint32)])
    c32, s32 = oracle_mod.sincos_turn(m, fp32=True)
    phi = 2.0 * np.pi * m.astype(np.float64) / 2.0 ** 24
    assert np.abs(c32 - np.cos(phi)).max() < 3e-7
    assert np.abs(s32 - np.sin(phi)).max() < 3e-7
    # quadrant points are exact
    c, s = oracle_mod.sincos_turn(np.array([0, 1 << 22, 1 << 23, 3 << 22], np.uint32), fp32=True)
    assert list(c) == [1.0, 0.0, -1.0, 0.0] and list(s) == [0.0, 1.0, 0.0, -1.0]


def test_onb_orthonormal(oracle_mod):
    rng = np.random.default_rng(3)
    n = rng.normal(size=(2000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n = np.concatenate([n, [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [0, 0.6, -0.8]]])
    b1, b2 = oracle_mod.onb(n)
    for a, b in [(b1, b1), (b2, b2), (n, n)]:
        assert np.abs((a * b).sum(1) - 1).max() < 1e-15 * 4
    for a, b in [(b1, b2), (b1, n), (b2, n)]:
        assert np.abs((a * b).sum(1)).max() < 1e-15 * 4


@pytest.mark.parametrize("normal", [(0, 0, 1), (0.3, -0.5, 0.812403840463596), (0.9, 0.1, -0.4242640687119285)])
def test_cosine_moments(oracle_mod, normal):
    n = np.array(normal, np.float64)
    n /= np.linalg.norm(n)
    N = 1 << 17
    rng = np.random.default_rng(5)
    x0 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
    x1 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
    d = oracle_mod.cosine_dirs(np.tile(n, (N, 1)), x0, x1, fp32=False)
    assert np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-14
    c = d @ n
    assert c.min() > 0
    # cos ~ sqrt(1-u1): mean 2/3, var 1/18; cos^2 ~ U: mean 1/2, var 1/12
    assert abs(c.mean() - 2 / 3) < 5 * np.sqrt(1 / 18 / N)
    assert abs((c * c).mean() - 0.5) < 5 * np.sqrt(1 / 12 / N)
    # tangential components average to zero
    t = d - np.outer(c, n)
    assert np.abs(t.mean(0)).max() < 5 * np.sqrt(0.5 / N)


def test_cosine_float_close_to_double(oracle_mod):
    rng = np.random.default_rng(9)
    N = 20000
    n = rng.normal(size=(N, 3))
    n[:, 2] = np.abs(n[:, 2])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n = n.astype(np.float32).astype(np.float64)
    x0 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
    x1 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
    d64 = oracle_mod.cosine_dirs(n, x0, x1, fp32=False)
    d32 = oracle_mod.cosine_dirs(n, x0, x1, fp32=True)
    assert np.abs(d64 - d32).max() < 2e-6
