"""Pins of the oracle's light-shared trace (one sample path per pixel and sample
serves all K lights) (no GPU).

Facts fixed outside the light-shared code:
* Its paths draw with light field 0, so light 0's estimate, its hit pixels and
  its shadow visibilities are exactly those of the per-light trace (pinned on its
  own) for light 0, for any bounce count and with or without shadow rays.
* A flat plane under a constant environment E: Lbar = E exactly for every light.
* Zero albedo: nothing depends on the light any more (every k is identical), and
  a black environment gives exactly 0.
* With a black environment, Lbar(k) is the sum over the recorded hits of the
  throughput product times rho * max(0, n.l_k) * V_k (recomputed from records).
* The estimator is unbiased like the per-light one: over independent seeds the
  two means agree within their standard errors for every light.
"""
import numpy as np
import pytest

import scenes


def _plane(H=10, W=12, albedo=0.6, C=1):
    depth = np.zeros((H, W), np.float32)
    normals = np.zeros((H, W, 3), np.float32)
    normals[..., 2] = 1.0
    return depth, normals, np.full((C, H, W), albedo, np.float32)


@pytest.mark.parametrize("B,shadow", [(1, True), (2, True), (3, True), (2, False)])
def test_light_zero_is_the_per_light_trace(oracle_mod, B, shadow):
    sc = scenes.mixed(31, 19, 23, K=5, C=3)
    args = (sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 12, B, 9, 2)
    a, ra, _ = oracle_mod.trace(*args, records=True, shadow_rays=shadow)
    b, rb, cb = oracle_mod.trace(*args, records=True, shadow_rays=shadow, shared=True)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(ra[:, 0, :, :, 0], rb[..., 0])  # hit pixels of every (pixel, sample, bounce)
    assert np.array_equal(ra[:, 0, :, :, 1], rb[..., 1])  # light 0's visibility
    assert (rb[..., 0] >= 0).sum() > 50
    # the other lights see the same hits with their own visibility
    assert not np.array_equal(a[1:], b[1:])
    assert cb[0] == sc.H * sc.W * 12


def test_flat_constant_env_exact(oracle_mod):
    d, n, a = _plane(C=3)
    E = np.array([0.2, 0.5, 0.125], np.float32)
    env = np.broadcast_to(E[:, None, None], (3, 4, 8)).copy()
    lights = np.asarray(scenes.ring_lights(4, 50.0), np.float32)
    lbar, rec, cnt = oracle_mod.trace(d, n, a, lights, env, 16, 2, 3, 5, shared=True, records=True)
    for c in range(3):
        assert np.all(lbar[:, c] == np.float64(E[c]))
    assert np.all(rec[..., 0, 0] == -1)
    assert cnt[0] == cnt[1] == 10 * 12 * 16  # one path per (pixel, sample), no shadow rays


def test_zero_albedo(oracle_mod):
    sc = scenes.bowl_64(20, 20, K=4)
    a0 = np.zeros_like(sc.albedo)
    lbar, _, _ = oracle_mod.trace(sc.depth, sc.normals, a0, sc.lights, np.zeros_like(sc.env), 16, 2, 1, 0,
                                  shared=True)
    assert np.all(lbar == 0.0)
    lbar, _, _ = oracle_mod.trace(sc.depth, sc.normals, a0, sc.lights, sc.env + 0.3, 16, 2, 1, 0, shared=True)
    for k in range(1, 4):
        assert np.array_equal(lbar[k], lbar[0])
    assert lbar.min() > 0.0


def test_black_env_equals_hit_sum(oracle_mod):
    sc = scenes.bowl_64(14, 14, K=3)
    albedo = np.stack([sc.albedo[0], 0.5 * sc.albedo[0] + 0.2]).astype(np.float32)
    black = np.zeros((2, 4, 8), np.float32)
    spp, B = 8, 3
    lbar, rec, _ = oracle_mod.trace(sc.depth, sc.normals, albedo, sc.lights, black, spp, B, 4, 1,
                                    records=True, shared=True)
    P, K = 14 * 14, 3
    nrm = sc.normals.reshape(P, 3).astype(np.float64)
    rho = albedo.reshape(2, P).astype(np.float64)
    L = sc.lights.astype(np.float64)
    want = np.zeros_like(lbar)
    for p in range(P):
        acc = np.zeros((K, 2))
        for s in range(spp):
            T = np.ones(2)
            for b in range(B):
                q = rec[p, s, b, 0]
                if q < 0:
                    break
                for k in range(K):
                    vis = rec[p, s, b, 1 + k]
                    if vis >= 0:
                        acc[k] += T * rho[:, q] * max(0.0, nrm[q] @ L[k]) * vis
                T = T * rho[:, q]
        want[:, :, p] = acc / spp
    assert np.abs(lbar - want).max() < 1e-14
    assert (rec[..., 0] >= 0).sum() > 100


def test_unbiased_like_per_light(oracle_mod):
    """Means over independent seeds of the two estimators agree for every light."""
    sc = scenes.mixed(44, 16, 16, K=4, C=1, n_bumps=2, n_bowls=2)
    env = sc.env[:1]
    per, sh = [], []
    for seed in range(10):
        a, _, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo[:1], sc.lights, env, 32, 2, 100 + seed, 0)
        b, _, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo[:1], sc.lights, env, 32, 2, 100 + seed, 0,
                                   shared=True)
        per.append(a[:, 0].mean(axis=1))
        sh.append(b[:, 0].mean(axis=1))
    per, sh = np.array(per), np.array(sh)
    se = np.sqrt(per.var(axis=0, ddof=1) / len(per) + sh.var(axis=0, ddof=1) / len(sh))
    assert np.all(np.abs(per.mean(axis=0) - sh.mean(axis=0)) <= 4.0 * se + 1e-12), (per.mean(0), sh.mean(0), se)
