"""Seeded synthetic scenes for IRT-PS (input generator only).

This module holds no step of the method: it draws ground-truth surfaces, their
analytic normals, albedo maps, light directions and environment maps.  Both the
oracle-side tests and the CUDA-side tests, benchmark and smoke check take their
inputs from here; neither the oracle nor the CUDA library imports it.

Conventions: an H x W heightfield sampled at pixel centres x_j = (j + 0.5) h,
y_i = (i + 0.5) h with h = 1 / W (object width 1); heights in the same unit;
normals n ~ (-dH/dx, -dH/dy, 1) from the analytic gradient; lights are unit
vectors with z > 0; the environment is a C x EH x EW latitude-longitude map over
the full sphere (theta = acos(w_z) down the rows, phi = atan2(w_y, w_x) across).

Workload recipes (stand-ins for the paper's synthetic, Harvard and face data,
which are not available):
  * `bowl_64`:   64x64 spherical-cap bowl (opening radius 0.4, depth 0.3),
                 albedo 0.7, constant grey environment 0.2, K = 8 lights at 45
                 degrees elevation, azimuths 2 pi k / 8.
  * `bumps_512`: 512x512, 20 Gaussian bumps/dents (amplitude U(-0.15, 0.15),
                 sigma U(0.02, 0.1)) plus a 90-degree V-groove (depth 0.1),
                 RGB albedo piecewise constant U(0.4, 0.9) over 16 Voronoi
                 cells, 32x64 RGB environment of 8 low-frequency cosines
                 (clamped >= 0), K = 12 lights at elevations U(30, 70) degrees.
  * `bumps_2048`: 2048x2048 RGB, 200 Gaussian bumps and 4 concave bowls
                 (opening radius U(0.05, 0.15), depth half the radius), 64x128
                 RGB cosine environment, K = 32 lights on a jittered ring
                 (azimuth 2 pi (k + U(-1/4, 1/4)) / K, elevation 45 +- U(-10, 10)
                 degrees); images stored in FP16.
  * `mixed`:     any size: bumps, bowls and grooves mixed at random (for ragged
                 and odd-sized test cases).
  * `bumps_4096`: 4096x4096 RGB, 1000 Gaussian bumps/dents (amplitude
                 U(-0.05, 0.05), sigma U(0.005, 0.03)) and 16 deep bowls (opening
                 radius U(0.03, 0.1), depth half the radius), 16-cell RGB Voronoi
                 albedo U(0.4, 0.9), 128x256 RGB cosine environment, K = 64 lights
                 on the jittered ring of `bumps_2048`.
  * `batch_objects`: the batched pattern: 64 objects of side
                 round(exp U(ln 96, ln 1024)) (square), K in {4, 8, 16, 32},
                 spp in {64, 128, 256}, bounces in {1, 2}, each a random mix of
                 bumps, bowls and a groove with RGB albedo U(0.3, 0.9).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    depth: np.ndarray      # (H, W) float32
    normals: np.ndarray    # (H, W, 3) float32, unit
    albedo: np.ndarray     # (C, H, W) float32
    lights: np.ndarray     # (K, 3) float32, unit, z > 0
    env: np.ndarray        # (C, EH, EW) float32
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def H(self):
        return self.depth.shape[0]

    @property
    def W(self):
        return self.depth.shape[1]

    @property
    def C(self):
        return self.albedo.shape[0]

    @property
    def K(self):
        return self.lights.shape[0]


def grid(H, W):
    h = 1.0 / W
    x = (np.arange(W) + 0.5) * h
    y = (np.arange(H) + 0.5) * h
    return np.meshgrid(x, y)  # X[i, j] = x_j, Y[i, j] = y_i


def normals_from_gradient(hx, hy):
    n = np.stack([-hx, -hy, np.ones_like(hx)], axis=-1)
    return n / np.linalg.norm(n, axis=-1, keepdims=True)


def ring_lights(K, elev_deg, az0=0.0):
    """K unit lights at the given elevation(s), azimuths az0 + 2 pi k / K."""
    el = np.radians(np.broadcast_to(np.asarray(elev_deg, np.float64), (K,)))
    az = az0 + 2.0 * np.pi * np.arange(K) / K
    return np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=1)


def bowl_field(X, Y, cx, cy, radius, depth):
    """Spherical-cap dent of opening radius `radius` and depth `depth`: (H, Hx, Hy)."""
    R = (radius ** 2 + depth ** 2) / (2.0 * depth)
    dx, dy = X - cx, Y - cy
    r2 = dx * dx + dy * dy
    inside = r2 < radius ** 2
    s = np.sqrt(np.maximum(R * R - r2, 1e-300))
    Hf = np.where(inside, (R - depth) - s, 0.0)
    Hx = np.where(inside, dx / s, 0.0)
    Hy = np.where(inside, dy / s, 0.0)
    return Hf, Hx, Hy


def gauss_field(X, Y, cx, cy, amp, sigma):
    e = amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sigma ** 2))
    return e, -e * (X - cx) / sigma ** 2, -e * (Y - cy) / sigma ** 2


def groove_field(X, Y, px, py, angle, depth):
    """90-degree V-groove (slopes +-1) of the given depth through (px, py)."""
    nx, ny = -np.sin(angle), np.cos(angle)
    s = (X - px) * nx + (Y - py) * ny
    inside = np.abs(s) < depth
    Hf = np.where(inside, np.abs(s) - depth, 0.0)
    sg = np.where(s >= 0, 1.0, -1.0)
    return Hf, np.where(inside, sg * nx, 0.0), np.where(inside, sg * ny, 0.0)


def voronoi_albedo(X, Y, rng, n_cells, C, lo, hi):
    seeds = np.stack([rng.uniform(0, X.max() + X.min(), n_cells),
                      rng.uniform(0, Y.max() + Y.min(), n_cells)], axis=1)
    vals = rng.uniform(lo, hi, (n_cells, C))
    d2 = (X[..., None] - seeds[:, 0]) ** 2 + (Y[..., None] - seeds[:, 1]) ** 2
    cell = np.argmin(d2, axis=-1)  # ties go to the lower seed index
    return np.moveaxis(vals[cell], -1, 0)


def cosine_env(rng, C, EH, EW, base=0.2, n_terms=8, amp=0.1):
    """max(0, base + sum_m a_mc cos(f_m theta + g_m phi + psi_m)), f, g in {0..3}."""
    th = (np.arange(EH) + 0.5) * np.pi / EH
    ph = (np.arange(EW) + 0.5) * 2.0 * np.pi / EW
    T, P = np.meshgrid(th, ph, indexing="ij")
    f = rng.integers(0, 4, n_terms)
    g = rng.integers(0, 4, n_terms)
    psi = rng.uniform(0, 2 * np.pi, n_terms)
    a = rng.uniform(0, amp, (n_terms, C))
    env = np.full((C, EH, EW), base)
    for m in range(n_terms):
        env += a[m][:, None, None] * np.cos(f[m] * T + g[m] * P + psi[m])[None]
    return np.maximum(env, 0.0)


def _finish(Hf, Hx, Hy, albedo, lights, env, name, **meta):
    return Scene(depth=np.asarray(Hf, np.float32),
                 normals=np.asarray(normals_from_gradient(Hx, Hy), np.float32),
                 albedo=np.asarray(albedo, np.float32),
                 lights=np.asarray(lights / np.linalg.norm(lights, axis=1, keepdims=True), np.float32),
                 env=np.asarray(env, np.float32), name=name, meta=meta)


def bowl_64(H=64, W=64, albedo=0.7, env_value=0.2, K=8, elev=45.0):
    """Concave spherical bowl (opening radius 0.4, depth 0.3), one channel."""
    X, Y = grid(H, W)
    Hf, Hx, Hy = bowl_field(X, Y, 0.5, 0.5 * H / W, 0.4, 0.3)
    return _finish(Hf, Hx, Hy, np.full((1, H, W), albedo), ring_lights(K, elev),
                   np.full((1, 4, 8), env_value), f"bowl_{H}x{W}")


def bumps_512(seed=2, H=512, W=512, K=12, n_bumps=20):
    """Gaussian bumps and dents + V-groove, Voronoi RGB albedo, cosine environment."""
    rng = np.random.default_rng(seed)
    X, Y = grid(H, W)
    Hf = np.zeros((H, W))
    Hx = np.zeros((H, W))
    Hy = np.zeros((H, W))
    ymax = H / W
    for _ in range(n_bumps):
        e, ex, ey = gauss_field(X, Y, rng.uniform(0, 1), rng.uniform(0, ymax), rng.uniform(-0.15, 0.15),
                                rng.uniform(0.02, 0.1))
        Hf += e
        Hx += ex
        Hy += ey
    e, ex, ey = groove_field(X, Y, rng.uniform(0.25, 0.75), rng.uniform(0.25, 0.75) * ymax,
                             rng.uniform(0, np.pi), 0.1)
    Hf += e
    Hx += ex
    Hy += ey
    albedo = voronoi_albedo(X, Y, rng, 16, 3, 0.4, 0.9)
    env = cosine_env(rng, 3, 32, 64)
    lights = ring_lights(K, rng.uniform(30.0, 70.0, K))
    return _finish(Hf, Hx, Hy, albedo, lights, env, f"bumps_{H}x{W}")


def _add_windowed_gauss(Hf, Hx, Hy, h, cx, cy, amp, sigma, reach=7.0):
    """Add a Gaussian bump evaluated within reach*sigma of its centre (beyond it the
    bump is below exp(-24.5) of its amplitude and is left out)."""
    H, W = Hf.shape
    j0 = max(0, int((cx - reach * sigma) / h - 0.5))
    j1 = min(W, int((cx + reach * sigma) / h + 1.5))
    i0 = max(0, int((cy - reach * sigma) / h - 0.5))
    i1 = min(H, int((cy + reach * sigma) / h + 1.5))
    if j0 >= j1 or i0 >= i1:
        return
    x = (np.arange(j0, j1) + 0.5) * h
    y = (np.arange(i0, i1) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    e, ex, ey = gauss_field(X, Y, cx, cy, amp, sigma)
    Hf[i0:i1, j0:j1] += e
    Hx[i0:i1, j0:j1] += ex
    Hy[i0:i1, j0:j1] += ey


def _voronoi_lowmem(X, Y, rng, n_cells, C, lo, hi):
    """voronoi_albedo computed seed by seed (ties to the lower seed index)."""
    seeds = np.stack([rng.uniform(0, X.max() + X.min(), n_cells),
                      rng.uniform(0, Y.max() + Y.min(), n_cells)], axis=1)
    vals = rng.uniform(lo, hi, (n_cells, C))
    best = np.full(X.shape, np.inf)
    cell = np.zeros(X.shape, np.int64)
    for m in range(n_cells):
        d2 = (X - seeds[m, 0]) ** 2 + (Y - seeds[m, 1]) ** 2
        closer = d2 < best
        best = np.where(closer, d2, best)
        cell = np.where(closer, m, cell)
    return np.moveaxis(vals[cell], -1, 0)


def bumps_2048(seed=3, H=2048, W=2048, K=32, n_bumps=200, n_bowls=4):
    """Gaussian bumps + concave bowls, Voronoi RGB albedo, 64x128 environment, jittered light ring."""
    rng = np.random.default_rng(seed)
    h = 1.0 / W
    ymax = H / W
    Hf = np.zeros((H, W))
    Hx = np.zeros((H, W))
    Hy = np.zeros((H, W))
    for _ in range(n_bumps):
        _add_windowed_gauss(Hf, Hx, Hy, h, rng.uniform(0, 1), rng.uniform(0, ymax), rng.uniform(-0.15, 0.15),
                            rng.uniform(0.02, 0.1))
    X, Y = grid(H, W)
    for _ in range(n_bowls):
        r = rng.uniform(0.05, 0.15)
        e, ex, ey = bowl_field(X, Y, rng.uniform(0.15, 0.85), rng.uniform(0.15, 0.85) * ymax, r, 0.5 * r)
        Hf += e
        Hx += ex
        Hy += ey
    albedo = _voronoi_lowmem(X, Y, rng, 16, 3, 0.4, 0.9)
    env = cosine_env(rng, 3, 64, 128)
    az = 2.0 * np.pi * (np.arange(K) + rng.uniform(-0.25, 0.25, K)) / K
    el = np.radians(45.0 + rng.uniform(-10.0, 10.0, K))
    lights = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=1)
    return _finish(Hf, Hx, Hy, albedo, lights, env, f"bumps_{H}x{W}")


def _add_windowed_bowl(Hf, Hx, Hy, h, cx, cy, radius, depth):
    """Add a bowl evaluated on its bounding box only (it is zero outside its opening)."""
    H, W = Hf.shape
    j0, j1 = max(0, int((cx - radius) / h - 1)), min(W, int((cx + radius) / h + 2))
    i0, i1 = max(0, int((cy - radius) / h - 1)), min(H, int((cy + radius) / h + 2))
    if j0 >= j1 or i0 >= i1:
        return
    X, Y = np.meshgrid((np.arange(j0, j1) + 0.5) * h, (np.arange(i0, i1) + 0.5) * h)
    e, ex, ey = bowl_field(X, Y, cx, cy, radius, depth)
    Hf[i0:i1, j0:j1] += e
    Hx[i0:i1, j0:j1] += ex
    Hy[i0:i1, j0:j1] += ey


def _jittered_ring(rng, K):
    az = 2.0 * np.pi * (np.arange(K) + rng.uniform(-0.25, 0.25, K)) / K
    el = np.radians(45.0 + rng.uniform(-10.0, 10.0, K))
    return np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=1)


def bumps_4096(seed=5, H=4096, W=4096, K=64, n_bumps=1000, n_bowls=16):
    """Many small bumps and deep bowls at 4096x4096, 128x256 environment, K = 64 lights."""
    rng = np.random.default_rng(seed)
    h = 1.0 / W
    ymax = H / W
    Hf = np.zeros((H, W))
    Hx = np.zeros((H, W))
    Hy = np.zeros((H, W))
    for _ in range(n_bumps):
        _add_windowed_gauss(Hf, Hx, Hy, h, rng.uniform(0, 1), rng.uniform(0, ymax), rng.uniform(-0.05, 0.05),
                            rng.uniform(0.005, 0.03))
    for _ in range(n_bowls):
        r = rng.uniform(0.03, 0.1)
        _add_windowed_bowl(Hf, Hx, Hy, h, rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9) * ymax, r, 0.5 * r)
    X, Y = grid(H, W)
    albedo = _voronoi_lowmem(X, Y, rng, 16, 3, 0.4, 0.9)
    del X, Y
    env = cosine_env(rng, 3, 128, 256)
    return _finish(Hf, Hx, Hy, albedo, _jittered_ring(rng, K), env, f"bumps_{H}x{W}")


def mixed(seed, H, W, K=6, C=3, n_bumps=6, n_bowls=2, groove=True, EH=16, EW=32):
    """A random mix of Gaussian bumps, bowls and a groove at any size (test cases)."""
    rng = np.random.default_rng(seed)
    X, Y = grid(H, W)
    ymax = H / W
    Hf = np.zeros((H, W))
    Hx = np.zeros((H, W))
    Hy = np.zeros((H, W))
    for _ in range(n_bumps):
        e, ex, ey = gauss_field(X, Y, rng.uniform(0, 1), rng.uniform(0, ymax), rng.uniform(-0.12, 0.12),
                                rng.uniform(0.05, 0.15))
        Hf += e
        Hx += ex
        Hy += ey
    for _ in range(n_bowls):
        r = rng.uniform(0.1, 0.25)
        e, ex, ey = bowl_field(X, Y, rng.uniform(0.2, 0.8), rng.uniform(0.2, 0.8) * ymax, r, 0.5 * r)
        Hf += e
        Hx += ex
        Hy += ey
    if groove:
        e, ex, ey = groove_field(X, Y, rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7) * ymax,
                                 rng.uniform(0, np.pi), 0.06)
        Hf += e
        Hx += ex
        Hy += ey
    albedo = voronoi_albedo(X, Y, rng, 6, C, 0.3, 0.9)
    env = cosine_env(rng, C, EH, EW)
    lights = ring_lights(K, rng.uniform(35.0, 65.0, K), rng.uniform(0, 2 * np.pi))
    return _finish(Hf, Hx, Hy, albedo, lights, env, f"mixed_{H}x{W}")


def random_heightfield(seed, H, W, amp=0.2):
    """Rough random heights (for intersection tests), float32."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-amp, amp, (H, W))).astype(np.float32)


def plain_state(scene):
    """The ground truth as an estimate (depth, normals, albedo) in float32."""
    return scene.depth, scene.normals, scene.albedo


def batch_spec(seed=4, n=64, side_lo=96, side_hi=1024):
    """Sizes and trace settings of a batch: list of (scene seed, side, K, spp, bounces)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(round(np.exp(rng.uniform(np.log(side_lo), np.log(side_hi)))))
        K = int(rng.choice([4, 8, 16, 32]))
        spp = int(rng.choice([64, 128, 256]))
        bounces = int(rng.choice([1, 2]))
        out.append((1000 * seed + i, side, K, spp, bounces))
    return out


def batch_objects(seed=4, n=64, side_lo=96, side_hi=1024):
    """The scenes of batch_spec: list of (Scene, spp, bounces)."""
    out = []
    for s, side, K, spp, bounces in batch_spec(seed, n, side_lo, side_hi):
        rng = np.random.default_rng(s)
        sc = mixed(s, side, side, K=K, C=3, n_bumps=int(rng.integers(2, 9)), n_bowls=int(rng.integers(0, 3)),
                   groove=bool(rng.integers(0, 2)))
        out.append((sc, spp, bounces))
    return out
