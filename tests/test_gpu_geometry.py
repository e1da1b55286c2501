"""GPU geometry against the oracle, bit for bit (sampling and ray / mesh hits).

Integer decisions of the trace (hit or miss, hit triangle) are taken in FP32 on
both sides with the same operation order, so they must agree exactly; the
sampled directions they are built from must agree to the bit.
"""
import zlib

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def test_directions_bitwise(lib, oracle_mod):
    rng = np.random.default_rng(1)
    N = 200000
    n = rng.normal(size=(N, 3))
    n[: N // 2, 2] = np.abs(n[: N // 2, 2])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n = n.astype(np.float32)
    n[:8] = [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [0, 0.6, 0.8], [0.6, 0, -0.8], [0, 0, 1], [0, 0, 1]]
    x0 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
    x1 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
    x1[6], x1[7] = 1 << 30, 1 << 31  # quadrant points: exact zeros in the direction
    got = lib.irtps_probe_dirs(n, x0, x1)
    want = oracle_mod.cosine_dirs(n.astype(np.float64), x0, x1, fp32=True).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def _rays(depth, rng, n):
    H, W = depth.shape
    out = []
    for _ in range(n):
        i, j = rng.integers(0, H), rng.integers(0, W)
        d = rng.normal(size=3)
        d[2] = abs(d[2]) * rng.choice([1.0, -0.3])
        d[:2] *= W
        out.append([j, i, depth[i, j] + 1e-3 / W, *d])
    for _ in range(n):
        x, y = rng.uniform(0, W - 1), rng.uniform(0, H - 1)
        d = rng.normal(size=3)
        d[:2] *= W
        out.append([x, y, depth.max() + rng.uniform(-0.3, 0.3), *d])
    for _ in range(n // 8):  # grid-line and vertex-aimed rays
        i0, j0 = rng.integers(0, H), rng.integers(0, W)
        i1, j1 = rng.integers(0, H), rng.integers(0, W)
        out.append([j0, i0, depth[i0, j0] + 1e-3, 0.0, rng.choice([-1.0, 1.0]) * W, rng.uniform(-0.3, 0.3)])
        out.append([j0, i0, depth[i0, j0] + 1e-3, rng.choice([-1.0, 1.0]) * W, 0.0, rng.uniform(-0.3, 0.3)])
        if (i0, j0) != (i1, j1):
            o = np.array([j0, i0, depth[i0, j0] + 0.3])
            out.append([*o, *(np.array([j1, i1, depth[i1, j1]]) - o)])
    return np.array(out, np.float32)


def _grazing_only(depth, rays, tri, t_b, tri_b):
    """Rays where the walk's triangle differs from brute force over every triangle.  The walk reports
    the first hit among the cells the ray passes through; brute force can also admit, by FP32
    rounding in the triangle test, a hit on the far side of a cell edge that the ray runs along
    within rounding of it.  Such a hit lies outside its own cell, by less than 1e-5 of a cell.
    Returns the number of rays that differ; fails on any other difference."""
    Wc = depth.shape[1] - 1
    bad = np.nonzero(tri != tri_b)[0]
    for r in bad:
        assert tri_b[r] >= 0, (r, rays[r], tri[r], tri_b[r])
        cy, cx = divmod(int(tri_b[r]) // 2, Wc)
        q = rays[r, :3].astype(np.float64) + t_b[r] * rays[r, 3:].astype(np.float64)
        outside = max(cx - q[0], q[0] - (cx + 1), cy - q[1], q[1] - (cy + 1))
        assert 0.0 < outside < 1e-5, (r, rays[r], tri[r], tri_b[r], outside)
    return bad.size


@pytest.mark.parametrize("case", ["random16", "bowl64", "mixed_37x53", "bumps_200x137", "tiny_2x3"])
def test_rays_match_oracle_walk(lib, oracle_mod, case):
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    if case == "random16":
        depth = scenes.random_heightfield(3, 16, 16, 0.3 / 16)
    elif case == "bowl64":
        depth = scenes.bowl_64().depth
    elif case == "mixed_37x53":
        depth = scenes.mixed(4, 37, 53).depth
    elif case == "bumps_200x137":
        depth = scenes.mixed(9, 200, 137, n_bumps=12, n_bowls=4).depth
    else:
        depth = np.array([[0.1, -0.2, 0.05], [0.0, 0.3, -0.1]], np.float32)
    H, W = depth.shape
    rays = _rays(depth, rng, 3000)
    ctx = lib.Context(H, W, scenes.ring_lights(3, 45.0), np.zeros((1, 2, 2), np.float32))
    try:
        ctx.set_state(depth=depth)
        t, tri = ctx.probe_rays(rays)
    finally:
        ctx.close()
    t_o, tri_o = oracle_mod.intersect(depth, rays.astype(np.float64), fp32=True, brute=False)
    bad = np.nonzero(tri != tri_o)[0]
    assert bad.size == 0, (case, bad[:5], tri[bad[:5]], tri_o[bad[:5]])
    hit = tri >= 0
    assert np.array_equal(t[hit], t_o[hit].astype(np.float32))
    assert hit.sum() > 100
    if H * W <= 16 * 16:
        t_b, tri_b = oracle_mod.intersect(depth, rays.astype(np.float64), fp32=True, brute=True)
        assert _grazing_only(depth, rays, tri, t_b, tri_b) <= 2  # a rounding corner, not a pattern
