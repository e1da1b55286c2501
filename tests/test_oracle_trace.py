"""Pins of the oracle's reverted Monte-Carlo trace (Eq. 5-7) (no GPU).

Facts fixed outside the oracle:
* A flat plane under a black environment receives exactly zero indirect light.
* Zero albedo: the concavity part is exactly zero (black environment gives 0;
  a constant environment E gives E times the fraction of escaping paths).
* A flat plane under a constant environment E: every path escapes, so each
  sample returns E and the irradiance pi*Lbar is pi*E exactly.
* A plane under a theta-only environment: the mean matches an independent
  quadrature of the interpolated map against the cosine density, and the
  spread of independent per-pixel estimates shrinks as 1/sqrt(spp).
* More bounces never lower Lbar (the first bounce draws identical numbers), and
  with a black environment Lbar equals the sum over recorded hits of the
  throughput product c1*c2 times the direct term at each hit.
* Results do not depend on the thread count or on the pixel subset.
"""
import numpy as np
import pytest

import scenes


def _plane(H=12, W=12, height=0.0, albedo=0.6, C=1):
    depth = np.full((H, W), height, np.float32)
    normals = np.zeros((H, W, 3), np.float32)
    normals[..., 2] = 1.0
    return depth, normals, np.full((C, H, W), albedo, np.float32)


def _lights(K=3):
    return np.asarray(scenes.ring_lights(K, 50.0), np.float32)


def test_flat_black_is_zero(oracle_mod):
    d, n, a = _plane()
    env = np.zeros((1, 8, 16), np.float32)
    for fp32 in (True, False):
        lbar, rec, cnt = oracle_mod.trace(d, n, a, _lights(), env, 16, 2, 7, 0, fp32=fp32, records=True)
        assert np.all(lbar == 0.0)
        assert np.all(rec[..., 0, 0] == -1)  # every primary ray escapes
        assert cnt[0] == cnt[1] == 12 * 12 * 3 * 16


def test_flat_constant_env_exact(oracle_mod):
    d, n, a = _plane(C=3)
    E = np.array([0.2, 0.5, 0.125], np.float32)
    env = np.broadcast_to(E[:, None, None], (3, 4, 8)).copy()
    lbar, _, _ = oracle_mod.trace(d, n, a, _lights(), env, 32, 1, 3, 5)
    for c in range(3):
        assert np.all(lbar[:, c] == np.float64(E[c]))
    assert np.allclose(np.pi * lbar[:, 1], np.pi * 0.5, rtol=0, atol=0)


def test_zero_albedo(oracle_mod):
    sc = scenes.bowl_64(24, 24)
    a0 = np.zeros_like(sc.albedo)
    black = np.zeros_like(sc.env)
    lbar, _, _ = oracle_mod.trace(sc.depth, sc.normals, a0, sc.lights, black, 16, 2, 1, 0)
    assert np.all(lbar == 0.0)
    # constant environment: E times the escaping fraction, read from the records
    E = np.float32(0.3)
    env = np.full_like(sc.env, E)
    lbar, rec, _ = oracle_mod.trace(sc.depth, sc.normals, a0, sc.lights, env, 16, 2, 1, 0, records=True)
    esc = (rec[..., 0, 0] == -1)  # first bounce escapes: T = 1
    # (hits at bounce 1 carry T = rho = 0 afterwards, so only first-bounce escapes count)
    frac = esc.mean(axis=2)  # (P, K)
    assert np.allclose(lbar[:, 0, :], (np.float64(E) * frac).T, rtol=0, atol=1e-15)
    assert 0.05 < frac.mean() < 0.999  # the bowl does occlude part of the sky


def _theta_env(EH=16, EW=8):
    vals = 0.1 + 0.8 * np.linspace(0.0, 1.0, EH) ** 1.5  # any theta profile
    return np.repeat(vals[:, None], EW, axis=1)[None].astype(np.float32), vals


def _theta_expectation(vals, EH):
    """E[Env] under the cosine density about +z: 2 * int_0^{pi/2} Env(theta) cos sin dtheta,
    Env piecewise linear between texel centres (clamped), by Gauss-Legendre per piece."""
    centres = (np.arange(EH) + 0.5) * np.pi / EH
    knots = np.concatenate([[0.0], centres[(centres > 0) & (centres < np.pi / 2)], [np.pi / 2]])
    xg, wg = np.polynomial.legendre.leggauss(40)
    total = 0.0
    for lo, hi in zip(knots[:-1], knots[1:]):
        th = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
        f = np.interp(th, centres, vals.astype(np.float32).astype(np.float64))
        total += 0.5 * (hi - lo) * np.sum(wg * f * 2.0 * np.cos(th) * np.sin(th))
    return total


def test_theta_env_mean_and_inverse_sqrt_spp(oracle_mod):
    H = W = 20
    d, n, a = _plane(H, W)
    env, vals = _theta_env()
    exact = _theta_expectation(vals, env.shape[1])
    spreads = []
    for spp in [4, 16, 64, 256]:
        lbar, _, _ = oracle_mod.trace(d, n, a, _lights(1), env, spp, 1, 123, 0, threads=0)
        est = lbar[0, 0]  # H*W independent estimates (distinct pixel counters)
        sd = est.std(ddof=1)
        spreads.append(sd * np.sqrt(spp))
        # the pooled mean is unbiased: within 4 standard errors
        assert abs(est.mean() - exact) < 4 * sd / np.sqrt(est.size)
    spreads = np.array(spreads)
    # sd * sqrt(spp) is the single-sample spread: constant across spp (1/sqrt(N) rule)
    assert spreads.max() / spreads.min() < 1.25


def test_more_bounces_never_lower(oracle_mod):
    sc = scenes.mixed(3, 20, 17, K=3, C=3)
    l1, _, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 16, 1, 9, 2)
    l2, _, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 16, 2, 9, 2)
    l3, _, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 16, 3, 9, 2)
    assert np.all(l2 >= l1) and np.all(l3 >= l2)
    inc2 = (l2 - l1).sum()
    inc3 = (l3 - l2).sum()
    assert inc2 > 0 and inc3 < inc2  # deeper bounces contribute less (darker)


def test_black_env_equals_hit_sum(oracle_mod):
    """Recompute Lbar from the records: sum_b (prod_{b'<b} rho_{q_b'}) rho_{q_b} max(0, n_{q_b}.l) V."""
    sc = scenes.bowl_64(16, 16, K=3)
    albedo = np.stack([sc.albedo[0], 0.5 * sc.albedo[0] + 0.2]).astype(np.float32)
    black = np.zeros((2, 4, 8), np.float32)
    spp, B = 8, 3
    lbar, rec, _ = oracle_mod.trace(sc.depth, sc.normals, albedo, sc.lights, black, spp, B, 4, 1,
                                    records=True)
    P = 16 * 16
    nrm = sc.normals.reshape(P, 3).astype(np.float64)
    rho = albedo.reshape(2, P).astype(np.float64)
    L = sc.lights.astype(np.float64)
    want = np.zeros_like(lbar)
    for p in range(P):
        for k in range(3):
            acc = np.zeros(2)
            for s in range(spp):
                T = np.ones(2)
                for b in range(B):
                    q, vis = rec[p, k, s, b]
                    if q < 0:
                        break
                    if vis >= 0:
                        acc += T * rho[:, q] * max(0.0, nrm[q] @ L[k]) * vis
                    T = T * rho[:, q]
            want[k, :, p] = acc / spp
    assert np.abs(lbar - want).max() < 1e-14
    assert (rec[..., 0] >= 0).sum() > 100  # the bowl produces hits


def test_threads_and_subsets_agree(oracle_mod):
    sc = scenes.mixed(8, 18, 21, K=4, C=3)
    full, rec, cnt = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 8, 2, 77, 3,
                                      threads=1, records=True)
    multi, rec2, cnt2 = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 8, 2, 77, 3,
                                         threads=4, records=True)
    assert np.array_equal(full, multi) and np.array_equal(rec, rec2) and cnt == cnt2
    pix = np.array([0, 5, 17 * 21 - 1, 100, 101], np.int32)
    sub, recs, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 8, 2, 77, 3,
                                    pixels=pix, records=True)
    assert np.array_equal(sub, full[:, :, pix]) and np.array_equal(recs, rec[pix])
    # a different iteration index draws different numbers
    other, _, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 8, 2, 77, 4)
    assert not np.array_equal(other, full)


def test_double_and_float_geometry_agree(oracle_mod):
    sc = scenes.mixed(12, 24, 24, K=3, C=1)
    l64, r64, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 8, 2, 5, 0,
                                   fp32=False, records=True)
    l32, r32, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 8, 2, 5, 0,
                                   fp32=True, records=True)
    # decisions in the two precisions differ only on a tiny fraction of segments
    same = (r64[..., 0, :] == r32[..., 0, :]).all(-1)
    assert same.mean() > 0.999
    assert np.abs(l64 - l32).mean() < 1e-3
