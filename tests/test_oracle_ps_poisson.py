"""Pins of the oracle's photometric stereo (Eq. 3-4) and integration (no GPU).

* An analytic Lambertian convex sphere with no inter-reflection and no noise
  gives the normals back to 1e-9 rad (all rows valid, and with masked rows).
* Three orthogonal lights reduce Eq. 4 to n = normalize(A), rho = |A|.
* Fewer than 3 valid rows, or coplanar valid lights, mark the pixel invalid.
* Integration reproduces planes and paraboloids exactly (trapezoidal edge
  gradients are exact for quadratics), matches a dense least-squares solve of
  the edge system on small grids, and returns a mean-zero surface.
* Forward / inverse consistency: subtracting the very indirect estimate used to
  render the images leaves direct light plus noise, and PS recovers the
  ground-truth normals within the noise bound.
"""
import numpy as np
import pytest

import scenes


def _sphere(n=41):
    # convex cap of the unit sphere seen from +z, over [-0.8, 0.8]^2
    x = np.linspace(-0.8, 0.8, n)
    X, Y = np.meshgrid(x, x)
    inside = X ** 2 + Y ** 2 < 0.95 ** 2
    X, Y = X[inside], Y[inside]
    return np.stack([X, Y, np.sqrt(1.0 - X ** 2 - Y ** 2)], -1)


def test_sphere_exact(oracle_mod):
    N = _sphere()
    L = scenes.ring_lights(8, 60.0, 0.1)
    rho = 0.8
    A = rho * (N @ L.T).T  # (K, P), no clamp: keep the pixels lit by all lights
    lit = (A > 1e-3).all(axis=0)
    I = A[:, None, :]
    valid = np.ones((8, N.shape[0]), bool)
    n, r, ok = oracle_mod.ps_solve(I[:, :, lit], valid[:, lit], L)
    assert ok.all()
    err = np.radians(oracle_mod.angular_error_deg(n, N[lit]))
    assert err.max() < 1e-9
    assert np.abs(r - rho).max() < 1e-12
    # shadowed rows (n.l <= 0) clamped to zero and masked: still exact where >= 3 rows remain
    A2 = rho * np.maximum(0.0, (N @ L.T).T)
    v2 = A2 > 1e-6
    n2, r2, ok2 = oracle_mod.ps_solve(A2[:, None, :], v2, L)
    enough = v2.sum(axis=0) >= 3
    assert np.array_equal(ok2, enough)
    err2 = np.radians(oracle_mod.angular_error_deg(n2[ok2], N[ok2]))
    assert err2.max() < 1e-9
    assert (~v2).any(axis=0).sum() > 50  # the masked path was exercised


def test_three_orthogonal_lights(oracle_mod):
    rng = np.random.default_rng(2)
    L = np.eye(3)
    A = rng.uniform(0.05, 0.9, (3, 1, 500))
    n, r, ok = oracle_mod.ps_solve(A, np.ones((3, 500), bool), L)
    a = A[:, 0, :].T
    assert np.abs(n - a / np.linalg.norm(a, axis=1, keepdims=True)).max() < 1e-15
    assert np.abs(r[0] - np.linalg.norm(a, axis=1)).max() < 1e-15


def test_pinv_is_least_squares(oracle_mod):
    rng = np.random.default_rng(4)
    L = scenes.ring_lights(7, rng.uniform(30, 70, 7))
    A = rng.uniform(0, 1, (7, 20))
    G = oracle_mod.pinv_lights(L) @ A
    G2 = np.linalg.lstsq(L, A, rcond=None)[0]
    assert np.abs(G - G2).max() < 1e-13


def test_invalid_pixels(oracle_mod):
    L = scenes.ring_lights(6, 45.0)
    I = np.full((6, 1, 3), 0.3)
    valid = np.ones((6, 3), bool)
    valid[:4, 0] = False           # only 2 rows
    valid[:, 1] = False
    valid[[0, 3], 1] = True        # 2 rows (opposite lights)
    I[:, :, 2] = 0.0               # zero images: zero vector, undefined direction
    n, r, ok = oracle_mod.ps_solve(I, valid, L)
    assert not ok.any()
    assert np.all(n == [0.0, 0.0, 1.0]) and np.all(r == 0.0)
    # coplanar valid lights: all on one great circle through z -> rank 2 -> rejected by the condition number
    Lc = np.array([[1, 0, 1], [0.5, 0, 1], [-1, 0, 1], [0, 1, 1.0]])
    Lc /= np.linalg.norm(Lc, axis=1, keepdims=True)
    v = np.array([[True], [True], [True], [False]])
    n, r, ok = oracle_mod.ps_solve(np.full((4, 1, 1), 0.5), v, Lc)
    assert not ok[0]


def test_rgb_reduces_to_grey(oracle_mod):
    N = _sphere(21)
    L = scenes.ring_lights(6, 55.0)
    A = (N @ L.T).T
    rhos = np.array([0.2, 0.5, 0.9])
    I = rhos[None, :, None] * A[:, None, :]
    n, r, ok = oracle_mod.ps_solve(I, np.ones(A.shape, bool), L)
    assert np.radians(oracle_mod.angular_error_deg(n, N)).max() < 1e-9
    assert np.abs(r - rhos[:, None]).max() < 1e-12


def _normals_of(hx, hy):
    return scenes.normals_from_gradient(hx, hy)


@pytest.mark.parametrize("H,W", [(8, 8), (13, 21), (64, 48)])
def test_integrate_plane_and_paraboloid(oracle_mod, H, W):
    X, Y = scenes.grid(H, W)
    h = 1.0 / W
    for f, fx, fy in [
        (0.3 * X - 0.7 * Y, 0.3 + 0 * X, -0.7 + 0 * Y),
        (0.9 * (X ** 2 + Y ** 2) - 0.4 * X * Y, 1.8 * X - 0.4 * Y, 1.8 * Y - 0.4 * X),
    ]:
        Hs = oracle_mod.poisson_solve(_normals_of(fx, fy), h)
        want = f - f.mean()
        assert np.abs(Hs - want).max() < 1e-10 * max(1.0, np.ptp(want))
        assert abs(Hs.mean()) < 1e-13


def test_integrate_matches_dense_least_squares(oracle_mod):
    rng = np.random.default_rng(6)
    H, W = 7, 9
    n = rng.normal(size=(H, W, 3))
    n[..., 2] = np.abs(n[..., 2]) + 0.2
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    h = 1.0 / W
    p, q = oracle_mod.gradients(n)
    rows, g = [], []
    idx = np.arange(H * W).reshape(H, W)
    for i in range(H):
        for j in range(W - 1):
            r = np.zeros(H * W)
            r[idx[i, j + 1]] = 1
            r[idx[i, j]] = -1
            rows.append(r)
            g.append(h * (p[i, j] + p[i, j + 1]) / 2)
    for i in range(H - 1):
        for j in range(W):
            r = np.zeros(H * W)
            r[idx[i + 1, j]] = 1
            r[idx[i, j]] = -1
            rows.append(r)
            g.append(h * (q[i, j] + q[i + 1, j]) / 2)
    D = np.array(rows)
    x = np.linalg.lstsq(D, np.array(g), rcond=None)[0]  # minimum norm: mean zero
    Hs = oracle_mod.poisson_solve(n, h)
    assert np.abs(Hs.ravel() - x).max() < 1e-12
    # and it satisfies the normal equations
    b = oracle_mod.poisson_rhs(p, q, h)
    assert np.abs(oracle_mod.laplacian_apply(Hs) - b).max() < 1e-12


def test_nz_clamp(oracle_mod):
    n = np.array([[[0.0, 0.99, 0.01]]])
    p, q = oracle_mod.gradients(n)
    assert q[0, 0] == -0.99 / 0.05 and p[0, 0] == 0.0


def test_forward_inverse_consistency(oracle_mod):
    sc = scenes.bowl_64(32, 32)
    sigma = 0.002
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 32, 1, 11, sigma)
    K, C, H, W = A0.shape
    lbar, _, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 32, 1, 11,
                                  oracle_mod.FORWARD_ITER, stream=1)
    I = oracle_mod.correct_images(A0.reshape(K, C, -1), sc.albedo.reshape(C, -1), lbar)
    vis = oracle_mod.pixel_visibility(sc.depth, sc.normals, sc.lights).reshape(K, -1)
    n64 = sc.normals.reshape(-1, 3).astype(np.float64)
    direct = sc.albedo.reshape(1, -1).astype(np.float64) * np.maximum(0, n64 @ sc.lights.T.astype(np.float64)).T
    direct = np.where(vis == 1, direct, 0.0)
    z = oracle_mod.noise(H, W, C, K, 11).reshape(K, C, -1)
    # I = direct + sigma z up to the float32 rounding of the stored images
    assert np.abs(I[:, 0] - (direct + sigma * z[:, 0])).max() < 2e-7
    valid = oracle_mod.valid_rows(A0.reshape(K, C, -1), sc.albedo.reshape(C, -1), lbar)
    n, r, ok = oracle_mod.ps_solve(I, valid, sc.lights)
    lit = ok & (valid.sum(0) == K)
    err = np.radians(oracle_mod.angular_error_deg(n[lit], sc.normals.reshape(-1, 3)[lit]))
    bound = 6 * sigma * np.linalg.norm(oracle_mod.pinv_lights(sc.lights), 2) / 0.7
    assert lit.sum() > 300
    assert np.median(err) < bound / 3 and err.max() < bound
