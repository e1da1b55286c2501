"""Stage-wise parity of one IRT iteration on the GPU (helper of the loop tests).

From the GPU's own state before iteration t (surface H_t, normals n_t, albedo
rho_t), the oracle runs each stage of the iteration and every stage output of the
GPU must match it:

* trace (Sec. IV, Eq. 5-7): Lbar_t over the GPU's surface with the same Philox
  stream, within 1e-4 relative (of the image's largest value at holes when the
  single-sample variant fills them);
* subtract + PS (Eq. 4) from the GPU's own Lbar_t: row masks and validity
  bit-exact, normals within 1e-3 deg, albedo within 1e-5 of its range;
* integration of the GPU's normals n_{t+1}: H_{t+1} within 1e-4 of the depth
  range at every pixel (least squares, or the Huber M-estimator by IRLS);
* D_H between the GPU's two surfaces.

Feeding each stage the GPU's inputs keeps the comparison at the stated bars from
the first iteration to the last: a free-running comparison lets the two loops
drift apart through row masks that the FP32 and FP64 Lbar put on different sides
of tau_lo, and bounds the depth only in the mean."""
import numpy as np

from conftest import rel_close

LBAR_RTOL = 1e-4
NORMAL_MAX_DEG = 1e-3
DEPTH_MAX_OF_RANGE = 1e-4


def snapshot(ctx):
    """The GPU state the next iteration starts from."""
    return {"depth": ctx.depth(), "normals": ctx.normals(), "albedo": ctx.albedo(), "valid": ctx.valid()}


def check_iteration(oracle_mod, A0, lights, env, before, after, lbar, spp, bounces, seed, t, *, obj=0,
                    shared=False, irls=None, fill_holes=False, shadow_rays=True):
    """Check iteration t stage by stage; returns the oracle's D_H of the GPU's surfaces.
    before / after: snapshot() before and after the iteration; lbar: the GPU's Lbar_t
    (K, C, H, W); irls: (delta, reweighting steps) of robust integration, or None."""
    K, C, H, W = A0.shape
    P = H * W
    lb_o, rec, _ = oracle_mod.trace(before["depth"], before["normals"][..., :3], before["albedo"], lights, env,
                                    spp, bounces, seed, t, obj=obj, shared=shared, records=fill_holes,
                                    shadow_rays=shadow_rays)
    atol = 1e-7
    if fill_holes:
        known = ~oracle_mod.hole_mask(rec).reshape(K, H, W)
        lb_o = oracle_mod.interpolate_holes(lb_o.reshape(K, C, H, W), known).reshape(K, C, P)
        atol = LBAR_RTOL * float(np.abs(lb_o).max()) + 1e-7
    lb_g = np.asarray(lbar, np.float64).reshape(K, C, P)
    ok, worst = rel_close(lb_g, lb_o, LBAR_RTOL, atol)
    assert ok, ("Lbar", t, worst)
    # subtract + PS from the GPU's Lbar and albedo
    n_o, rho_o, ok_o = oracle_mod.ps_step(np.asarray(A0, np.float32), before["albedo"].reshape(C, P), lb_g, lights)
    v = after["valid"].reshape(-1).astype(bool)
    assert np.array_equal(v, ok_o), ("row masks", t, int((v != ok_o).sum()))
    n_g = after["normals"][..., :3].reshape(-1, 3)
    if v.any():
        err = oracle_mod.angular_error_deg(n_g[v], n_o[v])
        assert err.max() < NORMAL_MAX_DEG, ("normals", t, float(err.max()))
    assert np.abs(after["albedo"].reshape(C, P) - rho_o).max() <= 1e-5 * max(1.0, float(rho_o.max())), ("albedo", t)
    # integration of the GPU's normals
    nn = after["normals"][..., :3].astype(np.float64)
    if irls is not None:
        want_d = oracle_mod.irls_solve(nn, 1.0 / W, irls[0], irls[1])
    else:
        want_d = oracle_mod.poisson_solve(nn, 1.0 / W)
    dmax = np.abs(after["depth"] - want_d).max() / np.ptp(want_d)
    assert dmax <= DEPTH_MAX_OF_RANGE, ("depth", t, float(dmax))
    return oracle_mod.diff_norm(after["depth"], before["depth"])[0]
