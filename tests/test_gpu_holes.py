"""Single-sample variant on the GPU (holes of the per-light trace and their
non-uniform interpolation) against the oracle.

* The interpolation entry point on seeded stacks (ragged, degenerate and
  bench-sized shapes, sparse to dense holes, images without known pixels):
  known pixels keep their bits; holes within 1e-5 of the image's value range
  (FP32 pull-push against FP64).
* A context with fill_holes: the hole mask of a whole-field trace equals the
  oracle's (bit for bit, from its segment records); Lbar equals the oracle's
  filled Lbar within the trace tolerance (1e-4 relative plus 1e-6 of the largest
  value at known pixels, 1e-4 of the image's largest value at holes, which blend
  many known pixels).
* The full 512x512, K = 12 single-sample launch the bench times, whole field.
* The loop with fill_holes against the oracle loop; options that cannot combine
  with it are refused.
"""
import numpy as np
import pytest

import scenes
from conftest import rel_close
from stagewise import check_iteration, snapshot

pytestmark = pytest.mark.gpu

RTOL = 1e-4


def _stack(seed, K, C, H, W, p_hole):
    rng = np.random.default_rng(seed)
    v = rng.uniform(-0.5, 1.5, (K, C, H, W)).astype(np.float32)
    holes = (rng.random((K, H, W)) < p_hole).astype(np.uint8)
    return v, holes


def _check_fill(oracle_mod, got, v, holes, want=None):
    if want is None:
        want = oracle_mod.interpolate_holes(v, holes == 0)
    known = holes == 0
    for k in range(v.shape[0]):
        for c in range(v.shape[1]):
            g, w = got[k, c], want[k, c]
            assert np.array_equal(g[known[k]], v[k, c][known[k]]), (k, c)
            span = max(float(np.ptp(v[k, c][known[k]])) if known[k].any() else 0.0, 1e-30)
            err = float(np.abs(g - w).max()) if g.size else 0.0
            assert err <= 1e-5 * max(span, float(np.abs(w).max())), (k, c, err, span)


@pytest.mark.parametrize("K,C,H,W,p", [
    (1, 1, 1, 1, 1.0), (2, 3, 1, 9, 0.6), (3, 1, 7, 1, 0.5), (1, 3, 2, 2, 0.25), (4, 3, 13, 22, 0.7),
    (2, 1, 64, 64, 0.95), (3, 3, 97, 131, 0.3), (2, 3, 33, 17, 0.0), (2, 1, 40, 24, 0.999)])
def test_interpolation_matches_oracle(lib, oracle_mod, K, C, H, W, p):
    v, holes = _stack(1000 + H * W + K, K, C, H, W, p)
    if K > 1:
        holes[0] = 1  # an image without known pixels stays as it is
    got = lib.irtps_interpolate_holes(v, holes)
    _check_fill(oracle_mod, got, v, holes)
    if K > 1:
        assert np.array_equal(got[0], v[0])


def test_interpolation_bench_sized_stack(lib, oracle_mod):
    """512 x 512, K = 12, C = 3, 90 % holes: the size of the bench's Lbar."""
    v, holes = _stack(7, 12, 3, 512, 512, 0.9)
    got = lib.irtps_interpolate_holes(v, holes)
    _check_fill(oracle_mod, got, v, holes)


def test_interpolation_rejects_bad_arguments(lib):
    v, holes = _stack(8, 2, 3, 4, 5, 0.5)
    with pytest.raises(lib.IrtpsError) as e:
        lib.irtps_interpolate_holes(v.reshape(2, 3, 4, 5)[:, :2], holes)  # C = 2
    assert e.value.code == lib.IRTPS_EINVAL


def _fill_ctx(lib, sc):
    opt = lib.irtps_default_options()
    opt.fill_holes = 1
    ctx = lib.Context(sc.H, sc.W, sc.lights, sc.env, opt)
    ctx.set_state(sc.depth, sc.normals, sc.albedo)
    return ctx


def _compare_filled(oracle_mod, sc, got, holes, spp, bounces, seed, it, threads=0):
    want_raw, rec, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, spp, bounces, seed, it,
                                        fp32=True, records=True, threads=threads)
    want_holes = oracle_mod.hole_mask(rec)
    assert np.array_equal(holes.reshape(sc.K, -1), want_holes.astype(np.uint8))
    known = ~want_holes
    want = oracle_mod.interpolate_holes(want_raw.reshape(sc.K, sc.C, sc.H, sc.W),
                                        known.reshape(sc.K, sc.H, sc.W)).reshape(sc.K, sc.C, -1)
    g = got.reshape(sc.K, sc.C, -1)
    kk = np.broadcast_to(known[:, None, :], g.shape)
    if kk.any():
        # one sample per value: no average hides the FP32 rounding of a path, so the
        # absolute floor is FP32 resolution at the image's scale
        ok, worst = rel_close(g[kk], want[kk], RTOL, 1e-6 * float(np.abs(want).max()))
        assert ok, worst
    for k in range(sc.K):
        for c in range(sc.C):
            span = float(np.abs(want[k, c]).max()) + 1e-6
            assert np.abs(g[k, c] - want[k, c]).max() <= RTOL * span, (k, c)
    return want_holes


CASES = {
    "bowl64_c1": lambda: scenes.bowl_64(),
    "mixed_45x38_c3": lambda: scenes.mixed(31, 45, 38, K=5, C=3),
    "mixed_33x70_c1": lambda: scenes.mixed(32, 33, 70, K=3, C=1, n_bowls=3),
    "smallest_2x2": lambda: scenes.mixed(34, 2, 2, K=3, C=1),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("spp,bounces", [(1, 2), (1, 3), (4, 1)])
def test_context_marks_and_fills_holes(lib, oracle_mod, case, spp, bounces):
    sc = CASES[case]()
    seed, it = 0xABCDEF, 3
    with _fill_ctx(lib, sc) as ctx:
        ctx.trace(spp, bounces, seed, it)
        got = ctx.indirect()
        holes = ctx.holes()
        st = ctx.stats()
    assert st["walk_overflows"] == 0
    h = _compare_filled(oracle_mod, sc, got, holes, spp, bounces, seed, it)
    if sc.H * sc.W > 4:
        assert 0 < h.mean() < 1


def test_flat_plane_all_holes_keeps_traced_values(lib):
    """Every ray from a plane rises and leaves: all holes, no known pixel, so Lbar
    stays the traced environment radiance."""
    sc = scenes.mixed(35, 12, 16, K=4, C=3)
    sc.depth[:] = 0.0
    sc.normals[:] = (0.0, 0.0, 1.0)
    with _fill_ctx(lib, sc) as ctx, lib.Context(sc.H, sc.W, sc.lights, sc.env) as plain:
        ctx.trace(1, 2, 5, 0)
        plain.set_state(sc.depth, sc.normals, sc.albedo)
        plain.trace(1, 2, 5, 0)
        assert ctx.holes().all()
        assert np.array_equal(ctx.indirect(), plain.indirect())


def test_full_size_single_sample_bench_launch(lib, oracle_mod):
    """512 x 512 RGB bumps, K = 12, one sample per (pixel, light), 2 bounces: the
    whole field of the bench's single-sample launch against the oracle."""
    sc = scenes.bumps_512()
    spp, bounces, seed, it = 1, 2, 1, 0
    with _fill_ctx(lib, sc) as ctx:
        ctx.trace(spp, bounces, seed, it)
        got = ctx.indirect()
        holes = ctx.holes()
        assert ctx.stats()["walk_overflows"] == 0
    h = _compare_filled(oracle_mod, sc, got, holes, spp, bounces, seed, it)
    assert 0.05 < h.mean() < 0.99


def test_loop_with_holes_matches_oracle_loop(lib, oracle_mod):
    sc = scenes.mixed(36, 40, 44, K=6, C=3)
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 32, 2, 3, 0.002)
    spp, bounces, seed, n_iter = 1, 2, 17, 2
    hist = oracle_mod.irtps_run(A0, sc.lights, sc.env, n_iter, spp, bounces, seed, fill_holes=True)
    opt = lib.irtps_default_options()
    opt.fill_holes = 1
    with lib.Context(sc.H, sc.W, sc.lights, sc.env, opt) as ctx:
        ctx.set_images(A0)
        for t in range(n_iter):
            before = snapshot(ctx)
            ctx.iterate(1, spp, bounces, seed)
            st = ctx.stats()
            assert st["walk_overflows"] == 0 and st["cg_rel_residual"] <= 1e-9
            check_iteration(oracle_mod, A0, sc.lights, sc.env, before, snapshot(ctx), ctx.indirect(), spp, bounces,
                            seed, t, fill_holes=True)
            h = hist[t + 1]
            err = oracle_mod.angular_error_deg(ctx.normals()[..., :3].reshape(-1, 3), h["normals"].reshape(-1, 3))
            dabs = np.abs(ctx.depth() - h["depth"]) / np.ptp(h["depth"])
            assert err.mean() <= 0.05 and dabs.mean() <= 1e-4 and dabs.max() <= 1e-3, (t, err.mean(), dabs.max())


def test_graph_replay_fills_holes_the_same(lib, oracle_mod):
    sc = scenes.mixed(37, 30, 26, K=4, C=3)
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 16, 2, 3, 0.002)
    out = []
    for graph in (0, 1):
        opt = lib.irtps_default_options()
        opt.fill_holes = 1
        opt.use_graph = graph
        with lib.Context(sc.H, sc.W, sc.lights, sc.env, opt) as ctx:
            ctx.set_images(A0)
            ctx.iterate(3, 1, 2, 9)
            out.append((ctx.indirect(), ctx.holes(), ctx.normals()))
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_refusals(lib):
    sc = scenes.mixed(38, 10, 12, K=4, C=3)
    opt = lib.irtps_default_options()
    opt.fill_holes = 1
    opt.sampling = 1
    with pytest.raises(lib.IrtpsError) as e:
        lib.Context(sc.H, sc.W, sc.lights, sc.env, opt)
    assert e.value.code == lib.IRTPS_EINVAL
    with lib.Context(sc.H, sc.W, sc.lights, sc.env) as plain:
        with pytest.raises(lib.IrtpsError) as e:
            plain.holes()
        assert e.value.code == lib.IRTPS_EINVAL
    with _fill_ctx(lib, sc) as ctx:
        with pytest.raises(lib.IrtpsError) as e:
            lib.Batch([ctx])
        assert e.value.code == lib.IRTPS_EINVAL
