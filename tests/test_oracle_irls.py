"""Pins of the oracle's robust integration (Huber M-estimator by IRLS) (no GPU).

Facts fixed outside the IRLS code:
* With unit weights the sparse weighted solve equals the least-squares surface of
  the cosine-transform solution (two independent methods).
* A threshold above every residual leaves all weights at 1: IRLS = least squares.
* The weighted solution satisfies its normal equations, recomputed edge by edge.
* After enough reweighting steps the surface is a stationary point of the Huber
  objective: at every node the clipped residuals of its edges balance.
* Robustness: a block of corrupted normals spoils the least-squares surface around
  it; the Huber surface stays close to the truth outside the block.
"""
import numpy as np

import scenes


def _paraboloid(H=24, W=20, a=0.8):
    X, Y = scenes.grid(H, W)
    Hx, Hy = 2 * a * (X - 0.5), 2 * a * (Y - 0.5 * H / W)
    n = scenes.normals_from_gradient(Hx, Hy)
    d = a * ((X - 0.5) ** 2 + (Y - 0.5 * H / W) ** 2)
    return d - d.mean(), n


def test_unit_weights_equal_cosine_transform_solve(oracle_mod):
    sc = scenes.mixed(3, 21, 26, K=4, C=1)
    h = 1.0 / sc.W
    want = oracle_mod.poisson_solve(sc.normals, h)
    got = oracle_mod.weighted_poisson_solve(sc.normals, h, np.ones((sc.H, sc.W - 1)), np.ones((sc.H - 1, sc.W)))
    assert np.abs(got - want).max() <= 1e-10 * np.ptp(want)


def test_large_threshold_is_least_squares(oracle_mod):
    sc = scenes.mixed(4, 18, 15, K=4, C=1)
    h = 1.0 / sc.W
    want = oracle_mod.poisson_solve(sc.normals, h)
    got = oracle_mod.irls_solve(sc.normals, h, 1e6, 3)
    assert np.abs(got - want).max() <= 1e-10 * np.ptp(want)


def test_weighted_normal_equations(oracle_mod):
    rng = np.random.default_rng(5)
    sc = scenes.mixed(5, 13, 17, K=4, C=1)
    h = 1.0 / sc.W
    wh, wv = rng.uniform(0.1, 2.0, (13, 16)), rng.uniform(0.1, 2.0, (12, 17))
    d = oracle_mod.weighted_poisson_solve(sc.normals, h, wh, wv)
    p, q = oracle_mod.gradients(sc.normals)
    grad = np.zeros((13, 17))  # derivative of the weighted objective, edge by edge
    for i in range(13):
        for j in range(16):
            r = d[i, j + 1] - d[i, j] - h * (p[i, j] + p[i, j + 1]) / 2
            grad[i, j + 1] += wh[i, j] * r
            grad[i, j] -= wh[i, j] * r
    for i in range(12):
        for j in range(17):
            r = d[i + 1, j] - d[i, j] - h * (q[i, j] + q[i + 1, j]) / 2
            grad[i + 1, j] += wv[i, j] * r
            grad[i, j] -= wv[i, j] * r
    assert np.abs(grad).max() <= 1e-12
    assert abs(d.mean()) <= 1e-14


def test_huber_stationarity(oracle_mod):
    d_true, n = _paraboloid()
    rng = np.random.default_rng(6)
    n = n + rng.normal(0, 0.05, n.shape) * (rng.uniform(size=n.shape[:2]) < 0.1)[..., None]
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    H, W = n.shape[:2]
    h, delta = 1.0 / W, 0.05
    d = oracle_mod.irls_solve(n, h, delta, 60)
    uh, uv = oracle_mod.edge_slope_residuals(d, n, h)
    ph, pv = np.clip(uh, -delta, delta), np.clip(uv, -delta, delta)  # Huber influence psi(u)
    bal = np.zeros((H, W))
    bal[:, 1:] += ph
    bal[:, :-1] -= ph
    bal[1:, :] += pv
    bal[:-1, :] -= pv
    assert np.abs(bal).max() <= 1e-4 * delta
    assert (np.abs(uh) > delta).any()  # some edges are down-weighted


def test_corrupted_block_is_ignored(oracle_mod):
    d_true, n = _paraboloid(32, 32)
    bad = n.copy()
    bad[10:14, 12:16] = np.array([0.6, -0.5, 0.62]) / np.linalg.norm([0.6, -0.5, 0.62])
    h = 1.0 / 32
    ls = oracle_mod.poisson_solve(bad, h)
    rob = oracle_mod.irls_solve(bad, h, 0.05, 10)
    mask = np.ones((32, 32), bool)
    mask[8:16, 10:18] = False  # away from the block and its rim
    e_ls = np.abs((ls - ls[mask].mean()) - (d_true - d_true[mask].mean()))[mask].mean()
    e_rob = np.abs((rob - rob[mask].mean()) - (d_true - d_true[mask].mean()))[mask].mean()
    assert e_rob < 0.3 * e_ls, (e_rob, e_ls)
