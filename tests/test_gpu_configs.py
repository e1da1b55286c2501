"""Workload-sized GPU checks: the benchmark configuration at full size, FP16 input
images, the 2048x2048 K=32 configuration on sampled pixels, and the paper's
qualitative claim (IRT-PS r1..r3 against classic PS)."""
import numpy as np
import pytest

import scenes
from conftest import rel_close

pytestmark = pytest.mark.gpu


def test_bench_config_iteration0_full_size(lib, oracle_mod):
    """512x512 RGB bumps, K = 12: classic PS and integration over every pixel."""
    sc = scenes.bumps_512()
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 1, 1, 7, 0.002, indirect=False)
    K, C, H, W = A0.shape
    with lib.Context(H, W, sc.lights, sc.env) as ctx:
        ctx.set_images(A0)
        n, d, v = ctx.normals(), ctx.depth(), ctx.valid()
    want_n, _, ok = oracle_mod.ps_step(A0, np.zeros((C, H * W)), np.zeros((K, C, H * W)), sc.lights)
    assert np.array_equal(v.ravel().astype(bool), ok)
    err = oracle_mod.angular_error_deg(n[..., :3].reshape(-1, 3), want_n)
    assert err.mean() <= 0.05 and err[ok].max() < 1e-3
    want_d = oracle_mod.poisson_solve(want_n.reshape(H, W, 3), 1.0 / W)
    assert np.abs(d - want_d).max() <= 1e-4 * np.ptp(want_d)


def test_bench_config_loop_properties(lib):
    """The benchmark's job (GPU-rendered images, 256 spp, 2 bounces, 5 iterations): properties
    that hold at any size."""
    import torch
    sc = scenes.bumps_512()
    K, C, H, W = sc.K, sc.C, sc.H, sc.W
    with lib.Context(H, W, sc.lights, sc.env) as ctx:
        A0 = torch.empty((K, C, H, W), dtype=torch.float32, device="cuda")
        ctx.set_state(sc.depth, sc.normals, sc.albedo)
        ctx.render(256, 2, 1000, 0.002, out=A0)
        torch.cuda.synchronize()
        ctx.set_images(A0, on_device=True)
        dh = []
        for _ in range(5):
            dh.append(ctx.iterate(1, 256, 2, 1))
            st = ctx.stats()
            assert st["walk_overflows"] == 0 and st["cg_rel_residual"] <= 1e-9
        n, d, lb = ctx.normals(), ctx.depth(), ctx.indirect()
    nn = np.linalg.norm(n[..., :3], axis=-1)
    assert np.abs(nn - 1).max() < 1e-5
    assert abs(float(d.astype(np.float64).mean())) < 1e-6 * np.ptp(d)
    assert np.isfinite(lb).all() and lb.min() >= 0.0
    assert dh[-1] < dh[0]  # the loop settles


def test_fp16_images_loop(lib, oracle_mod):
    """Images stored in FP16: the GPU loop against the oracle loop fed the same FP16 values."""
    sc = scenes.mixed(51, 48, 40, K=8, C=3)
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 64, 2, 3, 0.002)
    A16 = A0.astype(np.float16)
    hist = oracle_mod.irtps_run(A16.astype(np.float32), sc.lights, sc.env, 2, 16, 2, 5)
    with lib.Context(sc.H, sc.W, sc.lights, sc.env) as ctx:
        ctx.set_images(A16, lib.IRTPS_F16)
        n0 = ctx.normals()
        ctx.iterate(2, 16, 2, 5)
        n2, d2 = ctx.normals(), ctx.depth()
    e0 = oracle_mod.angular_error_deg(n0[..., :3].reshape(-1, 3), hist[0]["normals"].reshape(-1, 3))
    e2 = oracle_mod.angular_error_deg(n2[..., :3].reshape(-1, 3), hist[2]["normals"].reshape(-1, 3))
    assert e0.mean() <= 0.05 and e2.mean() <= 0.05
    rng = np.ptp(hist[2]["depth"])
    assert np.abs(d2 - hist[2]["depth"]).mean() <= 1e-4 * rng


def test_config_2048_sampled_trace(lib, oracle_mod):
    """2048x2048 RGB, 200 bumps + 4 bowls, K = 32, 512 spp, 2 bounces: the full launch, checked
    on 64 sampled pixels (the four corners among them) that the oracle traces one by one."""
    sc = scenes.bumps_2048()
    spp, bounces, seed, it = 512, 2, 3, 0
    rng = np.random.default_rng(2)
    corners = [0, sc.W - 1, (sc.H - 1) * sc.W, sc.H * sc.W - 1]  # the grid's ragged edges
    pix = np.unique(np.concatenate([rng.choice(sc.H * sc.W, 60, replace=False), corners])).astype(np.int32)
    with lib.Context(sc.H, sc.W, sc.lights, sc.env) as ctx:
        ctx.set_state(sc.depth, sc.normals, sc.albedo)
        ctx.trace(spp, bounces, seed, it)
        st = ctx.stats()
        full = ctx.indirect().reshape(sc.K, sc.C, -1)[:, :, pix]
        sub, rec = ctx.trace_pixels(pix, spp, bounces, seed, it, records=True)
    want, rec_o, _ = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, spp, bounces, seed, it,
                                      pixels=pix, fp32=True, records=True)
    assert st["walk_overflows"] == 0
    assert np.array_equal(full, sub)
    assert np.array_equal(rec, rec_o)
    ok, worst = rel_close(full, want, 1e-4, 1e-7)
    assert ok, worst


def test_paper_trend_r1_r2_r3(lib, oracle_mod):
    """The claim of Table 1 and its discussion, on the concave bowl rendered with three
    reflections: IRT-PS with 1, 2 and 3 traced reflections each lowers the height and albedo
    errors (the paper's Eq. 8-9) and the normal error (Eq. 10) below classic PS."""
    sc = scenes.bowl_64()
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 256, 3, 11, 0.002)
    errs = {}
    for r in (1, 2, 3):
        with lib.Context(sc.H, sc.W, sc.lights, sc.env) as ctx:
            ctx.set_images(A0)
            if r == 1:
                errs["ps"] = (oracle_mod.height_error(sc.depth, ctx.depth()),
                              oracle_mod.albedo_error(sc.albedo, ctx.albedo()),
                              oracle_mod.normal_error(sc.normals, ctx.normals()[..., :3]))
            ctx.iterate(3, 64, r, 11)
            errs[r] = (oracle_mod.height_error(sc.depth, ctx.depth()),
                       oracle_mod.albedo_error(sc.albedo, ctx.albedo()),
                       oracle_mod.normal_error(sc.normals, ctx.normals()[..., :3]))
    for r in (1, 2, 3):
        for m in range(3):
            assert errs[r][m] < errs["ps"][m], (r, m, errs)
