"""Pins of the oracle's ray / heightfield intersection (no GPU).

* The triangle test agrees with an independent plane-and-barycentric solve.
* The cell walk agrees with brute force over every triangle of the mesh, hit for
  hit (triangle index and t), on heightfields of 16x16 or smaller: random, bowl,
  V-groove and plane, with random rays and adversarial ones (through vertices,
  along grid lines, grazing ridges), in both precisions.
"""
import numpy as np
import pytest

import scenes


def _plane_solve(o, d, v0, v1, v2):
    """Solve o + t d = v0 + u (v1 - v0) + v (v2 - v0) by a 3x3 linear solve."""
    M = np.stack([-d, v1 - v0, v2 - v0], axis=1)
    t, u, v = np.linalg.solve(M, o - v0)
    return t, u, v


def test_triangle_test_matches_linear_solve(oracle_mod):
    rng = np.random.default_rng(1)
    rows, expect = [], []
    while len(rows) < 3000:
        v0, v1, v2 = rng.uniform(-1, 1, (3, 3))
        o = rng.uniform(-1, 1, 3) + np.array([0, 0, 2])
        a, b = rng.uniform(-0.3, 1.0, 2)  # aim near the triangle: about half the rays hit
        d = v0 + a * (v1 - v0) + b * (v2 - v0) - o
        d *= rng.choice([1.0, -1.0], p=[0.9, 0.1]) / np.linalg.norm(d)
        try:
            t, u, v = _plane_solve(o, d, v0, v1, v2)
        except np.linalg.LinAlgError:
            continue
        margin = min(abs(u), abs(v), abs(1 - u - v), abs(t))
        if margin < 1e-6:
            continue  # keep clear of edges: the two formulas round differently there
        rows.append(np.concatenate([o, d, v0, v1, v2]))
        expect.append(t if (u >= 0 and v >= 0 and u + v <= 1 and t > 0) else np.nan)
    got = oracle_mod.tri_hit(np.array(rows), fp32=False)
    expect = np.array(expect)
    assert np.array_equal(np.isnan(got), np.isnan(expect))
    hit = ~np.isnan(expect)
    assert hit.sum() > 100
    assert np.abs(got[hit] - expect[hit]).max() < 1e-12


def test_vertical_ray_on_flat_cell(oracle_mod):
    depth = np.full((4, 5), 0.25, np.float32)
    rays = np.array([[1.3, 2.6, 1.0, 0.0, 0.0, -1.0]])
    for fp32 in (False, True):
        for brute in (False, True):
            t, tri = oracle_mod.intersect(depth, rays, fp32=fp32, brute=brute)
            assert t[0] == 0.75
            # (x, y) = (1.3, 2.6): cell (2, 1), below the diagonal -> T1 (y - 2 > x - 1)
            assert tri[0] == 2 * (2 * 4 + 1) + 1


def _fields():
    X, Y = scenes.grid(16, 16)
    bowl, _, _ = scenes.bowl_field(X, Y, 0.5, 0.5, 0.4, 0.3)
    groove, _, _ = scenes.groove_field(X, Y, 0.45, 0.55, 0.7, 0.2)
    return {
        "random16": scenes.random_heightfield(4, 16, 16, 0.3),
        "random_9x13": scenes.random_heightfield(5, 9, 13, 0.2),
        "bowl16": (bowl * 16).astype(np.float32),     # steep in grid units
        "groove16": (groove * 16).astype(np.float32),
        "plane": np.full((7, 11), -0.1, np.float32),
        "tilted": ((np.arange(12)[None, :] * 0.3 + np.arange(10)[:, None] * -0.2)).astype(np.float32),
    }


def _rays(depth, rng, n):
    H, W = depth.shape
    out = []
    # random origins inside the mesh extent, random directions (the trace only
    # starts rays at vertices or at hit points, never outside the mesh)
    for _ in range(n):
        x, y = rng.uniform(0, W - 1), rng.uniform(0, H - 1)
        z = depth.max() + rng.uniform(-0.5, 0.5) * (np.ptp(depth) + 0.1)
        d = rng.normal(size=3)
        out.append([x, y, z, *d])
    # from vertices (as the primary rays do), lifted slightly
    for _ in range(n):
        i, j = rng.integers(0, H), rng.integers(0, W)
        d = rng.normal(size=3)
        d[2] = abs(d[2]) * rng.choice([1, -0.3])
        out.append([j, i, depth[i, j] + 1e-3 / W, *d])
    # aimed exactly at vertices from vertices, along grid lines, grazing
    for _ in range(n // 4):
        i0, j0, i1, j1 = rng.integers(0, H), rng.integers(0, W), rng.integers(0, H), rng.integers(0, W)
        if (i0, j0) == (i1, j1):
            continue
        o = np.array([j0, i0, depth[i0, j0] + 0.5])
        tgt = np.array([j1, i1, depth[i1, j1]])
        out.append([*o, *(tgt - o)])
        out.append([j0, i0, depth[i0, j0] + 1e-3, 0.0, rng.choice([-1.0, 1.0]), rng.uniform(-0.3, 0.3)])
        out.append([j0, i0, depth[i0, j0] + 1e-3, rng.choice([-1.0, 1.0]), 0.0, rng.uniform(-0.3, 0.3)])
        # grazing: level ray just above the highest vertex, from inside a cell
        out.append([min(j0, W - 2) + 0.5, min(i0, H - 2) + 0.25, depth.max() + 1e-6, rng.normal(), rng.normal(),
                    0.0])
    return np.array(out, np.float64)


@pytest.mark.parametrize("fp32", [False, True])
def test_walk_equals_brute_force(oracle_mod, fp32):
    rng = np.random.default_rng(11)
    total_hits = 0
    for name, depth in _fields().items():
        rays = _rays(depth, rng, 600)
        t1, i1 = oracle_mod.intersect(depth, rays, fp32=fp32, brute=False)
        t2, i2 = oracle_mod.intersect(depth, rays, fp32=fp32, brute=True)
        bad = np.nonzero(i1 != i2)[0]
        assert bad.size == 0, (name, rays[bad[:5]], i1[bad[:5]], i2[bad[:5]])
        hit = i1 >= 0
        assert np.array_equal(t1[hit], t2[hit]), name
        total_hits += hit.sum()
    assert total_hits > 1000


def test_grazing_ray_walk_keeps_its_row(oracle_mod):
    """A ray from a vertex running within 1e-7 of a grid line: the cell walk tests the row the ray
    travels through (its hit lies inside its cell); brute force over every triangle also admits, by
    FP32 rounding in the triangle test, a hit in the neighbouring row 7.5e-8 of a cell outside that
    triangle's cell.  The walk's answer is the geometric one; the GPU reproduces the walk."""
    import scenes
    depth = scenes.random_heightfield(3, 16, 16, 0.3 / 16)
    ray = np.array([[11.0, 7.0, 0.011806140653789043, -1.0778954029083252, 0.0004152927431277931,
                     -0.3501964509487152]], np.float32).astype(np.float64)
    t_w, i_w = oracle_mod.intersect(depth, ray, fp32=True, brute=False)
    t_b, i_b = oracle_mod.intersect(depth, ray, fp32=True, brute=True)
    Wc = depth.shape[1] - 1

    def outside(t, i):
        cy, cx = divmod(int(i) // 2, Wc)
        q = ray[0, :3] + t * ray[0, 3:]
        return max(cx - q[0], q[0] - (cx + 1), cy - q[1], q[1] - (cy + 1))

    assert i_w[0] >= 0 and i_b[0] >= 0 and i_w[0] != i_b[0]
    assert outside(t_w[0], i_w[0]) <= 0.0          # the walk's hit: inside its own cell
    assert 0.0 < outside(t_b[0], i_b[0]) < 1e-6    # brute force's: a rounding hit across the edge
