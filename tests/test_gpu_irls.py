"""Robust integration (Huber M-estimator by IRLS) on the GPU against the oracle's
irls_solve: the same number of reweighting steps and threshold, both
preconditioners, ragged grids, a block of corrupted normals; and the whole loop
with robust integration against the oracle loop."""
import numpy as np
import pytest

import scenes
from stagewise import check_iteration, snapshot

pytestmark = pytest.mark.gpu


def _corrupted(seed, H, W):
    sc = scenes.mixed(seed, H, W, K=4, C=1)
    n = sc.normals.copy()
    i0, j0 = H // 3, W // 3
    n[i0:i0 + 4, j0:j0 + 5] = np.array([0.6, -0.5, 0.62], np.float32) / np.float32(np.linalg.norm([0.6, -0.5, 0.62]))
    return sc, n


@pytest.mark.parametrize("precond", [0, 1, 2])
@pytest.mark.parametrize("H,W,iters", [(33, 47, 3), (64, 64, 5), (2, 9, 2)])
def test_irls_integrate_matches_oracle(lib, oracle_mod, precond, H, W, iters):
    sc, n = _corrupted(90 + H, H, W)
    opt = lib.irtps_default_options()
    opt.precond = precond
    opt.irls_iters = iters
    opt.irls_delta = 0.05
    with lib.Context(H, W, sc.lights, sc.env, opt) as ctx:
        ctx.set_state(np.zeros((H, W), np.float32), n, sc.albedo)
        ctx.integrate()
        d = ctx.depth()
        st = ctx.stats()
        assert st["cg_rel_residual"] <= 1e-9
        n_used = ctx.normals()[..., :3]
    want = oracle_mod.irls_solve(n_used.astype(np.float64), 1.0 / W, 0.05, iters)
    assert np.abs(d - want).max() <= 1e-4 * np.ptp(want), np.abs(d - want).max() / np.ptp(want)
    ls = oracle_mod.poisson_solve(n_used.astype(np.float64), 1.0 / W)
    if H > 2:
        assert np.abs(want - ls).max() > 1e-3 * np.ptp(ls)  # the reweighting does change the surface


def test_irls_loop_matches_oracle(lib, oracle_mod):
    sc = scenes.mixed(97, 40, 44, K=6, C=3)
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 64, 2, 6, 0.002)
    hist = oracle_mod.irtps_run(A0, sc.lights, sc.env, 2, 16, 2, 5, irls_iters=3, irls_delta=0.05)
    opt = lib.irtps_default_options()
    opt.irls_iters = 3
    with lib.Context(sc.H, sc.W, sc.lights, sc.env, opt) as ctx:
        ctx.set_images(A0)
        out = [(ctx.normals(), ctx.depth())]
        for t in range(2):
            before = snapshot(ctx)
            ctx.iterate(1, 16, 2, 5)
            check_iteration(oracle_mod, A0, sc.lights, sc.env, before, snapshot(ctx), ctx.indirect(), 16, 2, 5, t,
                            irls=(0.05, 3))
            out.append((ctx.normals(), ctx.depth()))
    for t, ((n, d), h) in enumerate(zip(out, hist)):
        err = oracle_mod.angular_error_deg(n[..., :3].reshape(-1, 3), h["normals"].reshape(-1, 3))
        dabs = np.abs(d - h["depth"]) / np.ptp(h["depth"])
        assert err.mean() <= 0.05 and dabs.mean() <= 1e-4 and dabs.max() <= 1e-3, (t, err.mean(), dabs.max())
