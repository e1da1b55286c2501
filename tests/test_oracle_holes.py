"""Pins of the oracle's single-sample variant: hole mask and non-uniform hole interpolation (no GPU).

Facts fixed outside the code under test:
* Holes: from a flat surface every cosine-sampled ray rises and leaves, so every
  (pixel, light) is a hole; from the floor of a deep narrow pit almost every ray
  meets a wall, so almost none is; with a black environment a hole's radiance is
  exactly zero (its paths saw nothing).
* Interpolation (pull-push normalised convolution, the reading of the paper's
  unnamed non-uniform interpolation): known pixels keep their values bit for bit;
  a constant field is reproduced; one known pixel fills the whole image with its
  value; an image without known pixels is left as it is; every filled value is a
  convex combination of known values (within their range); mirrored inputs give
  mirrored outputs; channels do not mix; and three cases worked out by hand from the
  definition (1 x 4, 2 x 2, 3 x 3) fix the child sets of odd sizes and the
  upsampling weights 3/4, 1/4.
* Loop: with fill_holes the oracle loop's Lbar equals the plain trace at known
  pixels and the interpolation at holes.
"""
import numpy as np
import pytest

import scenes


def _rand(seed, K, C, H, W, p_known):
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1.0, 2.0, (K, C, H, W))
    known = rng.random((K, H, W)) < p_known
    return v, known


# ---------------------------------------------------------------- interpolation
def test_all_known_is_identity(oracle_mod):
    v, _ = _rand(1, 3, 2, 13, 22, 1.0)
    out = oracle_mod.interpolate_holes(v, np.ones((3, 13, 22), bool))
    assert np.array_equal(out, v)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (9, 1), (5, 6), (17, 33), (32, 32)])
def test_constant_field_reproduced(oracle_mod, shape):
    H, W = shape
    _, known = _rand(2, 2, 3, H, W, 0.3)
    known[:, 0, 0] = True
    v = np.full((2, 3, H, W), 0.37)
    v[0][:, ~known[0]] = 5.0  # garbage at holes must not leak
    v[1][:, ~known[1]] = -3.0
    out = oracle_mod.interpolate_holes(v, known)
    assert np.abs(out - 0.37).max() <= 1e-14


def test_single_known_pixel_fills_image(oracle_mod):
    K, C, H, W = 2, 3, 11, 14
    v = np.zeros((K, C, H, W))
    known = np.zeros((K, H, W), bool)
    known[0, 7, 3] = True
    known[1, 0, 13] = True
    v[0, :, 7, 3] = [0.25, -1.5, 3.0]
    v[1, :, 0, 13] = [2.0, 0.5, 1.0]
    out = oracle_mod.interpolate_holes(v, known)
    for k, (i, j) in enumerate([(7, 3), (0, 13)]):
        for c in range(C):
            assert np.abs(out[k, c] - v[k, c, i, j]).max() <= 1e-14


def test_no_known_pixel_leaves_image(oracle_mod):
    v, _ = _rand(3, 2, 3, 6, 9, 0.0)
    known = np.zeros((2, 6, 9), bool)
    known[1, 2, 2] = True
    out = oracle_mod.interpolate_holes(v, known)
    assert np.array_equal(out[0], v[0])
    assert np.abs(out[1] - v[1, :, 2:3, 2:3]).max() <= 1e-14


def test_hand_worked_1x4(oracle_mod):
    """[a, ?, ?, b]: level 1 is [a, b] (each coarse pixel has one known child), level 2
    (a + b) / 2 with confidence 1 leaves level 1 as it is; fine pixel 1 (odd) takes
    3/4 of coarse 0 and 1/4 of coarse 1, fine pixel 2 (even) 1/4 of coarse 0 and 3/4
    of coarse 1: [a, (3a + b) / 4, (a + 3b) / 4, b] = [2, 3, 5, 6] for a = 2, b = 6."""
    v = np.array([2.0, -9.0, 7.0, 6.0]).reshape(1, 1, 1, 4)
    known = np.array([True, False, False, True]).reshape(1, 1, 4)
    out = oracle_mod.interpolate_holes(v, known)
    assert np.array_equal(out.ravel(), [2.0, 3.0, 5.0, 6.0])


def test_hand_worked_2x2(oracle_mod):
    """One hole in a 2 x 2 image: the single coarse pixel is the mean of the three
    known values, and every fine pixel upsamples from it alone."""
    v = np.array([[1.0, 4.0], [-2.0, 0.0]]).reshape(1, 1, 2, 2)
    known = np.array([[True, True], [True, False]]).reshape(1, 2, 2)
    out = oracle_mod.interpolate_holes(v, known)
    assert out[0, 0, 1, 1] == pytest.approx(1.0, abs=1e-15)
    assert np.array_equal(out[0, 0][known[0]], v[0, 0][known[0]])


def test_hand_worked_3x3(oracle_mod):
    """Values 0..8 row-major with the centre missing.  Level 1 (2 x 2): top-left has
    the three known children 0, 1, 3 (mean 4/3); top-right the children 2, 5 (column
    3 does not exist; mean 3.5); bottom-left 6, 7 (6.5); bottom-right 8.  All four are
    fully confident, so the 1 x 1 level changes none of them.  The centre (odd row
    and column) takes weights 3/4 x 3/4, 3/4 x 1/4, 1/4 x 3/4, 1/4 x 1/4:
    0.5625 * 4/3 + 0.1875 * 3.5 + 0.1875 * 6.5 + 0.0625 * 8 = 3.125."""
    v = np.arange(9.0).reshape(1, 1, 3, 3)
    known = np.ones((1, 3, 3), bool)
    known[0, 1, 1] = False
    out = oracle_mod.interpolate_holes(v, known)
    assert out[0, 0, 1, 1] == pytest.approx(3.125, abs=1e-14)
    assert np.array_equal(out[0, 0][known[0]], v[0, 0][known[0]])


@pytest.mark.parametrize("seed,p", [(4, 0.05), (5, 0.3), (6, 0.8)])
def test_convex_and_known_pixels_kept(oracle_mod, seed, p):
    v, known = _rand(seed, 3, 3, 37, 29, p)
    known[:, 5, 5] = True
    out = oracle_mod.interpolate_holes(v, known)
    for k in range(3):
        for c in range(3):
            kv = v[k, c][known[k]]
            assert np.array_equal(out[k, c][known[k]], kv)
            assert out[k, c].min() >= kv.min() - 1e-12 and out[k, c].max() <= kv.max() + 1e-12


def test_mirror_symmetry_and_channel_independence(oracle_mod):
    v, known = _rand(7, 2, 3, 16, 32, 0.2)
    out = oracle_mod.interpolate_holes(v, known)
    flip = oracle_mod.interpolate_holes(v[..., ::-1], known[..., ::-1])
    assert np.abs(flip[..., ::-1] - out).max() <= 1e-13
    flip = oracle_mod.interpolate_holes(v[..., ::-1, :], known[..., ::-1, :])
    assert np.abs(flip[..., ::-1, :] - out).max() <= 1e-13
    v2 = v.copy()
    v2[:, 1] = 100.0 * v2[:, 1] + 3.0
    out2 = oracle_mod.interpolate_holes(v2, known)
    assert np.array_equal(out2[:, 0], out[:, 0]) and np.array_equal(out2[:, 2], out[:, 2])


def test_hole_far_from_data_is_smooth_blend(oracle_mod):
    """Two known pixels at opposite corners of a 1 x 8 row: every filled value lies
    between them and the row is monotone (no overshoot)."""
    v = np.zeros((1, 1, 1, 8))
    v[0, 0, 0, 0], v[0, 0, 0, 7] = -1.0, 3.0
    known = np.zeros((1, 1, 8), bool)
    known[0, 0, [0, 7]] = True
    out = oracle_mod.interpolate_holes(v, known).ravel()
    assert np.all(np.diff(out) >= -1e-15) and out[0] == -1.0 and out[7] == 3.0


# ---------------------------------------------------------------- hole mask
def _trace(oracle_mod, depth, normals, albedo, lights, env, spp, seed=11):
    return oracle_mod.trace(depth, normals, albedo, lights, env, spp, 2, seed, 0, records=True)


def test_flat_surface_every_pixel_is_a_hole(oracle_mod):
    H, W, K, C = 9, 12, 4, 3
    sc = scenes.mixed(21, H, W, K=K, C=C)
    depth = np.zeros((H, W), np.float32)
    normals = np.zeros((H, W, 3), np.float32)
    normals[..., 2] = 1.0
    env = np.zeros_like(sc.env)
    lbar, rec, _ = _trace(oracle_mod, depth, normals, sc.albedo, sc.lights, env, 3)
    holes = oracle_mod.hole_mask(rec)
    assert holes.shape == (K, H * W) and holes.all()
    assert np.all(lbar == 0.0)


def test_deep_pit_floor_is_almost_never_a_hole(oracle_mod):
    """A 3 x 3 floor five image-widths below its rim, 2/11 of a width across: a
    cosine-sampled ray escapes with probability below 1e-3, so of 8 lights x 9 floor
    pixels x 1 sample at most one (expected < 0.1) is a hole, while the flat rim
    around it, far from the pit, has holes."""
    H = W = 11
    K = 8
    sc = scenes.mixed(22, H, W, K=K, C=1)
    depth = np.zeros((H, W), np.float32)
    depth[4:7, 4:7] = -5.0
    normals = np.zeros((H, W, 3), np.float32)
    normals[..., 2] = 1.0
    _, rec, _ = _trace(oracle_mod, depth, normals, sc.albedo, sc.lights, sc.env, 1)
    holes = oracle_mod.hole_mask(rec).reshape(K, H, W)
    assert holes[:, 4:7, 4:7].sum() <= 1
    assert holes[:, 0, :].mean() > 0.5


def test_hole_radiance_is_zero_under_black_environment(oracle_mod):
    sc = scenes.mixed(23, 20, 17, K=5, C=3)
    env = np.zeros_like(sc.env)
    lbar, rec, _ = _trace(oracle_mod, sc.depth, sc.normals, sc.albedo, sc.lights, env, 1)
    holes = oracle_mod.hole_mask(rec)
    assert 0 < holes.sum() < holes.size
    assert np.all(lbar.transpose(1, 0, 2)[:, holes] == 0.0)
    assert np.all(rec[:, :, 0, 0, 0].T[~holes] >= 0)


# ---------------------------------------------------------------- loop
def test_loop_fills_holes_of_each_trace(oracle_mod):
    sc = scenes.mixed(24, 16, 18, K=4, C=3)
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 16, 2, 5, 0.002)
    hist = oracle_mod.irtps_run(A0, sc.lights, sc.env, 1, 1, 2, 9, fill_holes=True)
    st = hist[0]
    lbar, rec, _ = oracle_mod.trace(st["depth"].astype(np.float32), st["normals"].astype(np.float32),
                                    st["albedo"].astype(np.float32), sc.lights, sc.env, 1, 2, 9, 0, records=True)
    known = ~oracle_mod.hole_mask(rec)
    got = hist[1]["lbar"].reshape(4, 3, -1)
    assert 0 < known.sum() < known.size
    want = oracle_mod.interpolate_holes(lbar.reshape(4, 3, 16, 18), known.reshape(4, 16, 18)).reshape(4, 3, -1)
    assert np.array_equal(got, want)
    assert np.array_equal(got.transpose(1, 0, 2)[:, known], lbar.transpose(1, 0, 2)[:, known])
