"""The 4096x4096 RGB, K = 64 configuration at full size (1000 bumps, 16 deep bowls,
128x256 environment), FP16 and FP32 image storage on the same GPU, each checked
stage by stage against the oracle on a 512x512 crop given the GPU's own state:

* the trace of a full launch (iteration 0 state) on sampled crop pixels, which the
  oracle marches over the whole heightfield: records bit-exact, Lbar <= 1e-4;
* subtract + PS of the crop from the GPU's Lbar, albedo and images: row masks and
  validity bit-exact, normals within 0.05 deg;
* integration of the GPU's normals over the whole grid: within 1e-4 of the depth
  range of the exact cosine-transform solve.

The sample count is reduced (4 per pixel and light) to keep the test short; the
kernels, sizes and memory layout are those of the full configuration."""
import numpy as np
import pytest

import scenes
from conftest import rel_close

pytestmark = pytest.mark.gpu

SPP, B, SEED = 4, 2, 29
CROP = slice(1792, 2304)


@pytest.fixture(scope="module")
def scene():
    return scenes.bumps_4096()


def test_config5_fp16_and_fp32_against_oracle(lib, oracle_mod, scene):
    import torch
    sc = scene
    K, C, H, W = sc.K, sc.C, sc.H, sc.W
    A = torch.empty((K, C, H, W), dtype=torch.float32, device="cuda")
    with lib.Context(H, W, sc.lights, sc.env) as gt:
        gt.set_state(sc.depth, sc.normals, sc.albedo)
        gt.render(SPP, 1, 1000, 0.002, out=A)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    ci, cj = np.meshgrid(np.arange(H)[CROP], np.arange(W)[CROP], indexing="ij")
    crop_pix = (ci * W + cj).ravel()
    sample = np.sort(rng.choice(crop_pix, 64, replace=False)).astype(np.int32)
    normals_by = {}
    for name, dtype in (("f32", lib.IRTPS_F32), ("f16", lib.IRTPS_F16)):
        imgs = A if name == "f32" else A.half()
        with lib.Context(H, W, sc.lights, sc.env) as ctx:
            ctx.set_images(imgs, dtype, on_device=True)
            assert ctx.stats()["cg_rel_residual"] <= 1e-9
            d0, n0, al0 = ctx.depth(), ctx.normals(), ctx.albedo()
            sub, rec = ctx.trace_pixels(sample, SPP, B, SEED, 0, records=True)
            ctx.iterate(1, SPP, B, SEED)
            st = ctx.stats()
            assert st["walk_overflows"] == 0 and st["cg_rel_residual"] <= 1e-9
            n1, d1, v1 = ctx.normals(), ctx.depth(), ctx.valid()
            lb = torch.empty((K, C, H, W), dtype=torch.float32, device="cuda")
            ctx.indirect(out=lb)
            torch.cuda.synchronize()
            lb_crop = lb[:, :, CROP, CROP].reshape(K, C, -1).cpu().numpy()
            lb_sample = lb.reshape(K, C, -1)[:, :, torch.as_tensor(sample, device="cuda").long()].cpu().numpy()
            img_crop = imgs[:, :, CROP, CROP].float().cpu().numpy()
            del lb
        # trace: the iteration's full launch on the sampled pixels equals the per-pixel trace,
        # and both equal the oracle's march over the whole heightfield
        assert np.array_equal(lb_sample, sub)
        want, rec_o, _ = oracle_mod.trace(d0, n0[..., :3], al0, sc.lights, sc.env, SPP, B, SEED, 0,
                                          pixels=sample, records=True)
        assert np.array_equal(rec, rec_o)
        ok, worst = rel_close(sub, want, 1e-4, 1e-7)
        assert ok, worst
        # subtract + PS on the crop
        al0_crop = al0[:, CROP, CROP].reshape(C, -1)
        want_n, want_rho, ok_rows = oracle_mod.ps_step(img_crop, al0_crop, lb_crop, sc.lights)
        got_n = n1[CROP, CROP, :3].reshape(-1, 3)
        assert np.array_equal(v1[CROP, CROP].ravel().astype(bool), ok_rows)
        err = oracle_mod.angular_error_deg(got_n, want_n)
        assert err.mean() <= 0.05 and err[ok_rows].max() < 1e-3, (name, err.mean(), err.max())
        # integration of the GPU's normals over the whole grid
        want_d = oracle_mod.poisson_solve(n1[..., :3].astype(np.float64), 1.0 / W)
        assert np.abs(d1 - want_d).max() <= 1e-4 * np.ptp(want_d), name
        normals_by[name] = n1[CROP, CROP, :3].reshape(-1, 3)
    # FP16 storage changes the normals by the images' rounding only
    diff = oracle_mod.angular_error_deg(normals_by["f16"], normals_by["f32"])
    assert diff.mean() < 0.5, diff.mean()
