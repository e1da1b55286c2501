"""GPU reverted trace (Eq. 5-7) against the oracle.

Identical FP32 inputs on both sides (the ground-truth state of seeded scenes):
* every segment's record (hit pixel or escape, shadow visibility) is equal;
* Lbar agrees within 1e-4 relative (FP32 Kahan sums against FP64 sums);
* the full-image launch and the pixel-list launch agree bit for bit;
* runs are deterministic; the forward render matches the oracle's.
"""
import numpy as np
import pytest

import scenes
from conftest import rel_close

pytestmark = pytest.mark.gpu

RTOL = 1e-4


def _opts(lib, **kw):
    opt = lib.irtps_default_options()
    for k, v in kw.items():
        setattr(opt, k, v)
    return opt


def _ctx(lib, sc):
    ctx = lib.Context(sc.H, sc.W, sc.lights, sc.env)
    ctx.set_state(sc.depth, sc.normals, sc.albedo)
    return ctx


CASES = {
    "bowl64_c1": lambda: scenes.bowl_64(),
    "mixed_45x38_c3": lambda: scenes.mixed(21, 45, 38, K=5, C=3),
    "mixed_33x70_c1": lambda: scenes.mixed(22, 33, 70, K=3, C=1, n_bowls=3),
    "max_lights_16x12_k64": lambda: scenes.mixed(23, 16, 12, K=64, C=3),
    "smallest_2x2": lambda: scenes.mixed(24, 2, 2, K=3, C=1),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("spp,bounces", [(8, 2), (3, 3), (1, 1)])
def test_trace_records_and_lbar(lib, oracle_mod, case, spp, bounces):
    sc = CASES[case]()
    P = sc.H * sc.W
    pix = np.arange(P, dtype=np.int32)
    seed, it = 0x1234_5678_9ABC, 7
    with _ctx(lib, sc) as ctx:
        lbar, rec = ctx.trace_pixels(pix, spp, bounces, seed, it, records=True)
        ctx.trace(spp, bounces, seed, it)
        full = ctx.indirect().reshape(sc.K, sc.C, P)
        st = ctx.stats()
    want, rec_o, counts = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, spp, bounces, seed,
                                           it, fp32=True, records=True)
    bad = np.nonzero((rec != rec_o).any(axis=(-1, -2)))
    assert bad[0].size == 0, (case, [(int(a), int(b), int(c)) for a, b, c in zip(*bad)][:5])
    ok, worst = rel_close(lbar, want, RTOL, 1e-7)
    assert ok, (case, worst)
    assert np.array_equal(full, lbar)
    assert st["segments"] == counts[1] and st["primary_segments"] == counts[0]
    assert st["walk_overflows"] == 0
    if P > 4:
        assert (rec[..., 0] >= 0).mean() > 0.01  # some concavity hits


def test_trace_deterministic_and_seeded(lib):
    sc = scenes.mixed(5, 40, 40, K=4, C=3)
    with _ctx(lib, sc) as ctx:
        ctx.trace(16, 2, 99, 3)
        a = ctx.indirect()
        ctx.trace(16, 2, 99, 3)
        b = ctx.indirect()
        ctx.trace(16, 2, 99, 4)
        c = ctx.indirect()
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_flat_plane_constant_env(lib):
    H = W = 32
    depth = np.zeros((H, W), np.float32)
    normals = np.zeros((H, W, 3), np.float32)
    normals[..., 2] = 1
    albedo = np.full((3, H, W), 0.5, np.float32)
    E = np.array([0.2, 0.5, 0.125], np.float32)
    env = np.broadcast_to(E[:, None, None], (3, 8, 16)).copy()
    with lib.Context(H, W, scenes.ring_lights(4, 40.0), env) as ctx:
        ctx.set_state(depth, normals, albedo)
        ctx.trace(64, 2, 5, 0)
        lb = ctx.indirect()
    for c in range(3):
        assert np.abs(lb[:, c] - E[c]).max() <= 2e-7 * E[c]
    with lib.Context(H, W, scenes.ring_lights(4, 40.0), np.zeros_like(env)) as ctx:
        ctx.set_state(depth, normals, albedo)
        ctx.trace(64, 2, 5, 0)
        assert np.all(ctx.indirect() == 0.0)


def test_render_matches_oracle(lib, oracle_mod):
    sc = scenes.mixed(31, 41, 36, K=4, C=3)
    with _ctx(lib, sc) as ctx:
        img = ctx.render(16, 2, 77, 0.002)
    want = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 16, 2, 77, 0.002)
    assert np.abs(img - want).max() < 2e-5


def test_sampled_pixels_full_size_bench_launch(lib, oracle_mod):
    """512x512 RGB bumps, K=12, 256 spp, 2 bounces: the full launch the bench times,
    checked on sampled pixels the oracle traces one by one."""
    sc = scenes.bumps_512()
    spp, bounces, seed, it = 256, 2, 1, 0
    rng = np.random.default_rng(0)
    pix = np.sort(rng.choice(sc.H * sc.W, 48, replace=False)).astype(np.int32)
    with _ctx(lib, sc) as ctx:
        ctx.trace(spp, bounces, seed, it)
        full = ctx.indirect().reshape(sc.K, sc.C, -1)[:, :, pix]
        st = ctx.stats()
        sub, rec = ctx.trace_pixels(pix, spp, bounces, seed, it, records=True)
    want, rec_o, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, spp, bounces, seed, it,
                                      pixels=pix, fp32=True, records=True)
    assert st["walk_overflows"] == 0
    assert np.array_equal(full, sub)
    assert np.array_equal(rec, rec_o)
    ok, worst = rel_close(full, want, RTOL, 1e-7)
    assert ok, worst


def test_without_shadow_rays(lib, oracle_mod):
    """Option shadow_rays = 0: the direct term at a hit counts whenever n_q . l_k > 0."""
    sc = scenes.mixed(25, 31, 27, K=4, C=3)
    opt = lib.irtps_default_options()
    opt.shadow_rays = 0
    pix = np.arange(0, sc.H * sc.W, 7, dtype=np.int32)
    with lib.Context(sc.H, sc.W, sc.lights, sc.env, opt) as ctx:
        ctx.set_state(sc.depth, sc.normals, sc.albedo)
        lb, rec = ctx.trace_pixels(pix, 8, 2, 3, 1, records=True)
    want, rec_o, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 8, 2, 3, 1, pixels=pix,
                                      records=True, shadow_rays=False)
    assert np.array_equal(rec, rec_o)
    assert (rec[..., 1] == 0).sum() == 0  # nothing is ever shadowed
    ok, worst = rel_close(lb, want, RTOL, 1e-7)
    assert ok, worst


@pytest.mark.parametrize("case", ["mixed_45x38_c3", "mixed_33x70_c1", "bowl64_c1"])
def test_early_escape_keeps_every_bit(lib, oracle_mod, case):
    """The horizon test lets rising primary rays skip their march; records, Lbar and segment
    counts are those of the plain march, with fewer node visits."""
    sc = CASES[case]()
    out = []
    for early in (0, 1):
        opt = lib.irtps_default_options()
        opt.early_escape = early
        with lib.Context(sc.H, sc.W, sc.lights, sc.env, opt) as ctx:
            ctx.set_state(sc.depth, sc.normals, sc.albedo)
            lb, rec = ctx.trace_pixels(np.arange(sc.H * sc.W, dtype=np.int32), 16, 2, 5, 3, records=True)
            ctx.trace(16, 2, 5, 3)
            out.append((lb, rec, ctx.indirect(), ctx.stats()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
    assert out[0][3]["segments"] == out[1][3]["segments"]
    assert out[1][3]["node_visits"] < out[0][3]["node_visits"]


def test_early_escape_automatic_mode(lib):
    """Option 2 (the default) bounds horizons only for per-light traces of 16 or more
    samples per item over at least 2^18 work items; otherwise the trace runs without
    them.  Results never change."""
    sc = scenes.mixed(41, 160, 160, K=12, C=3)  # 307200 items
    res = {}
    for early in (0, 2):
        opt = lib.irtps_default_options()
        opt.early_escape = early
        with lib.Context(sc.H, sc.W, sc.lights, sc.env, opt) as ctx:
            ctx.set_state(sc.depth, sc.normals, sc.albedo)
            for spp in (8, 16):
                ctx.trace(spp, 2, 5, 3)
                res[early, spp] = (ctx.indirect(), ctx.stats()["node_visits"])
    assert lib.irtps_default_options().early_escape == 2
    for spp in (8, 16):
        assert np.array_equal(res[0, spp][0], res[2, spp][0])
    assert res[2, 8][1] == res[0, 8][1]
    assert res[2, 16][1] < res[0, 16][1]
    small = CASES["mixed_45x38_c3"]()  # 8550 items: left off
    with lib.Context(small.H, small.W, small.lights, small.env) as a, lib.Context(
            small.H, small.W, small.lights, small.env, _opts(lib, early_escape=0)) as b:
        for c in (a, b):
            c.set_state(small.depth, small.normals, small.albedo)
            c.trace(16, 2, 5, 3)
        assert a.stats()["node_visits"] == b.stats()["node_visits"]


def test_early_escape_keeps_every_bit_full_size(lib):
    """The bench's 512x512 surface: the whole field's Lbar and the records of a pixel
    sample are those of the plain march."""
    sc = scenes.bumps_512()
    rng = np.random.default_rng(3)
    pix = np.sort(rng.choice(sc.H * sc.W, 2048, replace=False)).astype(np.int32)
    out = []
    for early in (0, 1):
        opt = lib.irtps_default_options()
        opt.early_escape = early
        with lib.Context(sc.H, sc.W, sc.lights, sc.env, opt) as ctx:
            ctx.set_state(sc.depth, sc.normals, sc.albedo)
            lb, rec = ctx.trace_pixels(pix, 8, 2, 11, 1, records=True)
            ctx.trace(4, 2, 11, 1)
            out.append((lb, rec, ctx.indirect(), ctx.stats()))
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    assert out[0][3]["segments"] == out[1][3]["segments"]
    assert out[1][3]["node_visits"] < out[0][3]["node_visits"]
