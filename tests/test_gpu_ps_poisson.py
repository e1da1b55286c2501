"""GPU subtract + photometric stereo (Eq. 3-4) and depth integration against the oracle."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def _images(oracle_mod, sc, spp=16, bounces=1, seed=3, sigma=0.002):
    return oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, spp, bounces, seed, sigma)


@pytest.mark.parametrize("case", ["bowl64", "mixed_45x38_c3", "mixed_20x9_c3_k9"])
@pytest.mark.parametrize("f16", [False, True])
def test_ps_stage(lib, oracle_mod, case, f16):
    sc = {"bowl64": lambda: scenes.bowl_64(),
          "mixed_45x38_c3": lambda: scenes.mixed(8, 45, 38, K=6, C=3),
          "mixed_20x9_c3_k9": lambda: scenes.mixed(2, 20, 9, K=9, C=3)}[case]()
    A0 = _images(oracle_mod, sc)
    if f16:
        A0 = A0.astype(np.float16).astype(np.float32)
    K, C, H, W = A0.shape
    P = H * W
    rng = np.random.default_rng(1)
    lbar = (rng.uniform(0.0, 0.3, (K, C, P))).astype(np.float32)
    rho = (sc.albedo * rng.uniform(0.9, 1.1, sc.albedo.shape)).astype(np.float32)
    with lib.Context(H, W, sc.lights, sc.env) as ctx:
        ctx.set_images(A0.astype(np.float16) if f16 else A0, lib.IRTPS_F16 if f16 else lib.IRTPS_F32)
        n0, v0 = ctx.normals(), ctx.valid()
        ctx.set_state(albedo=rho)
        ctx.set_indirect(lbar.reshape(K, C, H, W))
        ctx.solve_normals()
        n1, a1, v1 = ctx.normals(), ctx.albedo(), ctx.valid()
    for (n, v, lb, r) in [(n0, v0, np.zeros_like(lbar), np.zeros((C, P))), (n1, v1, lbar, rho.reshape(C, P))]:
        want_n, want_r, ok = oracle_mod.ps_step(A0, r, lb, sc.lights)
        assert np.array_equal(v.ravel().astype(bool), ok)
        err = oracle_mod.angular_error_deg(n[..., :3].reshape(-1, 3)[ok], want_n[ok])
        assert err.max() < 1e-3, err.max()
        assert np.all(n[..., :3].reshape(-1, 3)[~ok] == [0, 0, 1])
    want_n, want_r, ok = oracle_mod.ps_step(A0, rho.reshape(C, P), lbar, sc.lights)
    assert np.abs(a1.reshape(C, P) - want_r).max() < 1e-5 * max(1.0, want_r.max())
    assert (~ok).sum() < P  # masked and valid pixels both present or all valid
    assert n1[..., 3].reshape(-1)[ok].min() > 0


def _cond1(M):
    return np.abs(M).sum(axis=1).max(axis=1) * np.abs(np.linalg.inv(M)).sum(axis=1).max(axis=1)


@pytest.mark.parametrize("f16", [False, True])
def test_ps_ill_conditioned_masked(lib, oracle_mod, f16):
    """Pixels that keep only a narrow arc of 3-6 of 12 lights (the rest in shadow): their masked
    systems are ill-conditioned (condition numbers far above 16), so the solve leaves the streaming
    pass for the list kernel (double-float matrix and re-read right-hand side, FP64 inverse).
    Masks and validity bit-exact, normals within 1e-3 deg and albedo within 1e-5 of the oracle, at
    iteration 0 and with an indirect term subtracted."""
    H, W, K, C = 37, 53, 12, 3
    P = H * W
    rng = np.random.default_rng(7)
    lights = scenes.ring_lights(K, rng.uniform(35.0, 55.0, K), az0=0.3)
    X, Y = scenes.grid(H, W)
    n = scenes.normals_from_gradient(0.4 * np.sin(9 * X + 2 * Y), 0.4 * np.cos(7 * Y - X)).reshape(P, 3)
    albedo = rng.uniform(0.4, 0.8, (C, P))
    shade = np.clip(n @ lights.T, 0.0, None).T  # K x P
    A0 = albedo[None] * shade[:, None, :] + rng.normal(0.0, 0.002, (K, C, P))
    keep = rng.integers(3, 7, P)
    start = rng.integers(0, K, P)
    arc = ((np.arange(K)[:, None] - start[None, :]) % K) < keep[None, :]
    arc[:, rng.uniform(size=P) < 0.2] = True  # some pixels keep every light
    A0 = np.where(arc[:, None, :], A0, 0.005).astype(np.float32)
    if f16:
        A0 = A0.astype(np.float16).astype(np.float32)
    lbar = rng.uniform(0.0, 0.02, (K, C, P)).astype(np.float32)
    rho = (albedo * rng.uniform(0.95, 1.05, albedo.shape)).astype(np.float32)
    env = np.zeros((C, 4, 8), np.float32)
    imgs = A0.reshape(K, C, H, W)
    with lib.Context(H, W, lights, env) as ctx:
        ctx.set_images(imgs.astype(np.float16) if f16 else imgs, lib.IRTPS_F16 if f16 else lib.IRTPS_F32)
        n0, a0, v0 = ctx.normals(), ctx.albedo(), ctx.valid()
        ctx.set_state(albedo=rho.reshape(C, H, W))
        ctx.set_indirect(lbar.reshape(K, C, H, W))
        ctx.solve_normals()
        n1, a1, v1 = ctx.normals(), ctx.albedo(), ctx.valid()
    L = np.asarray(lights, np.float32).astype(np.float64)
    for (nn, aa, vv, lb, r) in [(n0, a0, v0, np.zeros_like(lbar), np.zeros((C, P))),
                                (n1, a1, v1, lbar, rho)]:
        want_n, want_r, ok = oracle_mod.ps_step(imgs, r, lb, L)
        rows = oracle_mod.valid_rows(A0, r, lb, oracle_mod.TAU_LO, oracle_mod.TAU_HI)  # K x P
        masked = ok & ~rows.all(axis=0)
        M = np.einsum("kp,ki,kj->pij", rows[:, masked].astype(np.float64), L, L)
        assert (_cond1(M) > 16).sum() > 0.3 * P  # most pixels take the list kernel
        assert np.array_equal(vv.ravel().astype(bool), ok)
        err = oracle_mod.angular_error_deg(nn[..., :3].reshape(-1, 3)[ok], want_n[ok])
        assert err.max() < 1e-3, err.max()
        assert np.abs(aa.reshape(C, P)[:, ok] - want_r[:, ok]).max() < 1e-5 * max(1.0, want_r.max())


def test_ps_pinv_form_for_clustered_lights(lib, oracle_mod):
    """Lights in a narrow cone (L^T L with 1-norm condition number far above 16): fully valid pixels
    take the pinv(L) I form instead of the normal-equation form; parity as for the ring lights."""
    H, W, K, C = 29, 41, 8, 3
    P = H * W
    rng = np.random.default_rng(11)
    el = np.radians(rng.uniform(62.0, 72.0, K))
    az = rng.uniform(0.0, 0.8, K)
    lights = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=1)
    L = np.asarray(lights, np.float32).astype(np.float64)
    M = L.T @ L
    assert np.abs(M).sum(axis=0).max() * np.abs(np.linalg.inv(M)).sum(axis=0).max() > 16
    X, Y = scenes.grid(H, W)
    n = scenes.normals_from_gradient(0.3 * np.sin(5 * X), 0.3 * np.cos(4 * Y)).reshape(P, 3)
    albedo = rng.uniform(0.4, 0.8, (C, P))
    A0 = (albedo[None] * np.clip(n @ L.T, 0.0, None).T[:, None, :] + rng.normal(0.0, 0.002, (K, C, P)))
    A0 = A0.astype(np.float32)
    lbar = rng.uniform(0.0, 0.02, (K, C, P)).astype(np.float32)
    rho = (albedo * rng.uniform(0.95, 1.05, albedo.shape)).astype(np.float32)
    imgs = A0.reshape(K, C, H, W)
    with lib.Context(H, W, lights, np.zeros((C, 4, 8), np.float32)) as ctx:
        ctx.set_images(imgs, lib.IRTPS_F32)
        n0, a0, v0 = ctx.normals(), ctx.albedo(), ctx.valid()
        ctx.set_state(albedo=rho.reshape(C, H, W))
        ctx.set_indirect(lbar.reshape(K, C, H, W))
        ctx.solve_normals()
        n1, a1, v1 = ctx.normals(), ctx.albedo(), ctx.valid()
    for (nn, aa, vv, lb, r) in [(n0, a0, v0, np.zeros_like(lbar), np.zeros((C, P))),
                                (n1, a1, v1, lbar, rho)]:
        want_n, want_r, ok = oracle_mod.ps_step(imgs, r, lb, L)
        rows = oracle_mod.valid_rows(A0, r, lb, oracle_mod.TAU_LO, oracle_mod.TAU_HI)
        assert (ok & rows.all(axis=0)).sum() > P // 2  # mostly fully valid pixels
        assert np.array_equal(vv.ravel().astype(bool), ok)
        err = oracle_mod.angular_error_deg(nn[..., :3].reshape(-1, 3)[ok], want_n[ok])
        assert err.max() < 1e-3, err.max()
        assert np.abs(aa.reshape(C, P)[:, ok] - want_r[:, ok]).max() < 1e-5 * max(1.0, want_r.max())


@pytest.mark.parametrize("precond", [0, 1, 2])
@pytest.mark.parametrize("H,W", [(64, 64), (37, 53), (256, 256), (2, 5), (3, 301), (2, 1030)])
def test_integrate(lib, oracle_mod, H, W, precond):
    sc = scenes.mixed(H * 7 + W, H, W, K=3, C=1) if H > 3 else None
    rs = np.random.default_rng(H * W)
    normals = sc.normals if sc is not None else scenes.normals_from_gradient(
        rs.uniform(-0.3, 0.3, (H, W)), rs.uniform(-0.3, 0.3, (H, W))).astype(np.float32)
    lights = scenes.ring_lights(3, 45.0)
    opt = lib.irtps_default_options()
    opt.precond = precond
    with lib.Context(H, W, lights, np.zeros((1, 2, 2), np.float32), opt) as ctx:
        ctx.set_state(depth=np.zeros((H, W), np.float32), normals=normals)
        ctx.integrate()
        d = ctx.depth()
        st = ctx.stats()
    want = oracle_mod.poisson_solve(normals.astype(np.float64), 1.0 / W)
    rng = max(np.ptp(want), 1e-12)
    assert np.abs(d - want).max() <= 1e-4 * rng, (np.abs(d - want).max() / rng, st)
    assert abs(float(d.astype(np.float64).mean())) < 1e-6 * rng + 1e-9
    assert st["cg_rel_residual"] <= 1e-9


@pytest.mark.parametrize("H,W", [(2, 2), (17, 1024), (512, 512), (1024, 1024), (45, 38)])
def test_spectral_solve_is_direct(lib, oracle_mod, H, W):
    """precond = 2: one direct cosine-transform solve (the oracle's method, computed
    independently: FP64 transform products on the GPU, scipy's DCT on the host) lands
    within the FP32 rounding of the stored depth."""
    rs = np.random.default_rng(H + 3 * W)
    X, Y = scenes.grid(H, W)
    gx = 0.6 * np.sin(7 * X) * np.cos(5 * Y) + rs.normal(0, 0.05, (H, W))
    gy = 0.5 * np.cos(6 * X + 2 * Y) + rs.normal(0, 0.05, (H, W))
    normals = scenes.normals_from_gradient(gx, gy).astype(np.float32)
    opt = lib.irtps_default_options()
    assert opt.precond == 2
    with lib.Context(H, W, scenes.ring_lights(3, 45.0), np.zeros((1, 2, 2), np.float32), opt) as ctx:
        ctx.set_state(depth=np.zeros((H, W), np.float32), normals=normals)
        ctx.integrate()
        d = ctx.depth()
        st = ctx.stats()
    want = oracle_mod.poisson_solve(normals.astype(np.float64), 1.0 / W)
    rng = max(np.ptp(want), 1e-12)
    assert st["cg_iterations"] == 1 and st["cg_rel_residual"] <= 1e-10, st
    assert np.abs(d - want).max() <= 2e-6 * max(rng, np.abs(want).max()), np.abs(d - want).max() / rng


def test_integrate_quadric_exact(lib, oracle_mod):
    H, W = 96, 80
    X, Y = scenes.grid(H, W)
    f = 0.9 * (X ** 2 + Y ** 2) - 0.4 * X * Y + 0.2 * X
    n = scenes.normals_from_gradient(1.8 * X - 0.4 * Y + 0.2, 1.8 * Y - 0.4 * X).astype(np.float32)
    with lib.Context(H, W, scenes.ring_lights(3, 45.0), np.zeros((1, 2, 2), np.float32)) as ctx:
        ctx.set_state(depth=np.zeros((H, W), np.float32), normals=n)
        ctx.integrate()
        d = ctx.depth()
    want = f - f.mean()
    # exact up to the float32 rounding of the normals and of the stored depth
    assert np.abs(d - want).max() < 2e-5 * np.ptp(want)


@pytest.mark.parametrize("H,W", [(64, 48), (45, 38), (20, 9)])
def test_ps_widths_give_the_same_bits(lib, oracle_mod, H, W):
    """One, two or four pixels per thread (a tuning knob; grids whose pixel count is not a
    multiple fall back to one) and the tensor-core form's masks: the FP32 form's results do
    not depend on the width, bit for bit, through classic PS and a traced iteration."""
    sc = scenes.mixed(H + W, H, W, K=7, C=3)
    A0 = _images(oracle_mod, sc, spp=8)
    out = []
    for v in (1, 2, 4):
        with lib.Context(H, W, sc.lights, sc.env) as ctx:
            ctx.set_ps_tuning(v)
            assert ctx.ps_tuning() in ((v,) if (H * W) % v == 0 else (1,))
            ctx.set_images(A0.astype(np.float16), lib.IRTPS_F16)
            ctx.iterate(1, 4, 2, 3)
            out.append((ctx.normals(), ctx.albedo(), ctx.valid()))
    for o in out[1:]:
        for x, y in zip(out[0], o):
            assert np.array_equal(x, y)
