"""Light-shared sampling on the GPU against the oracle's light-shared trace: one
sample path per (pixel, sample) for all lights, a shadow ray per light at each hit.

Per-segment records (hit pixel, escape, each light's visibility) bit-exact; Lbar
within 1e-4 relative, whether a pixel's samples run as one work item or in chunks
(few traced pixels: many chunks); the whole loop against the oracle loop; a
graph-replayed iteration and other tuning give the same bits."""
import numpy as np
import pytest

import scenes
from conftest import rel_close
from stagewise import check_iteration, snapshot

pytestmark = pytest.mark.gpu


def _ctx(lib, sc, shadow=True, use_graph=0):
    opt = lib.irtps_default_options()
    opt.sampling = 1
    opt.shadow_rays = 1 if shadow else 0
    opt.use_graph = use_graph
    return lib.Context(sc.H, sc.W, sc.lights, sc.env, opt)


@pytest.mark.parametrize("seed,H,W,K,spp,B,shadow", [
    (81, 45, 38, 5, 16, 2, True), (82, 33, 70, 7, 8, 3, True), (83, 2, 3, 3, 32, 1, True),
    (84, 37, 53, 4, 12, 2, False)])
def test_trace_pixels_records_and_lbar(lib, oracle_mod, seed, H, W, K, spp, B, shadow):
    sc = scenes.mixed(seed, H, W, K=K, C=3)
    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(H * W, min(H * W, 40), replace=False)).astype(np.int32)
    with _ctx(lib, sc, shadow) as ctx:
        ctx.set_state(sc.depth, sc.normals, sc.albedo)
        lb, rec = ctx.trace_pixels(pix, spp, B, 7, 3, records=True)
        ctx.trace(spp, B, 7, 3)
        full = ctx.indirect().reshape(K, 3, -1)
        st = ctx.stats()
    want, rec_o, cnt = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, spp, B, 7, 3,
                                        pixels=pix, records=True, shadow_rays=shadow, shared=True)
    assert np.array_equal(rec.reshape(rec_o.shape), rec_o)
    ok, worst = rel_close(lb, want, 1e-4, 1e-7)
    assert ok, worst
    want_full, _, cnt_full = oracle_mod.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, spp, B, 7, 3,
                                              shadow_rays=shadow, shared=True)
    ok, worst = rel_close(full, want_full, 1e-4, 1e-7)
    assert ok, worst
    assert st["segments"] == cnt_full[1] and st["primary_segments"] == cnt_full[0]
    assert st["walk_overflows"] == 0


def test_shared_loop_matches_oracle(lib, oracle_mod):
    sc = scenes.mixed(85, 44, 40, K=6, C=3)
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 64, 2, 4, 0.002)
    hist = oracle_mod.irtps_run(A0, sc.lights, sc.env, 2, 24, 2, 11, shared=True)
    with _ctx(lib, sc) as ctx:
        ctx.set_images(A0)
        for t in range(2):
            before = snapshot(ctx)
            ctx.iterate(1, 24, 2, 11)
            check_iteration(oracle_mod, A0, sc.lights, sc.env, before, snapshot(ctx), ctx.indirect(), 24, 2, 11, t,
                            shared=True)
            n, d = ctx.normals(), ctx.depth()
            h = hist[t + 1]
            err = oracle_mod.angular_error_deg(n[..., :3].reshape(-1, 3), h["normals"].reshape(-1, 3))
            dabs = np.abs(d - h["depth"]) / np.ptp(h["depth"])
            assert err.mean() <= 0.05 and dabs.mean() <= 1e-4 and dabs.max() <= 1e-3, (t, err.mean(), dabs.max())
            st = ctx.stats()
            assert st["walk_overflows"] == 0 and st["cg_rel_residual"] <= 1e-9
            assert st["primary_segments"] == sc.H * sc.W * 24


def test_shared_graph_and_tuning_keep_bits(lib, oracle_mod):
    sc = scenes.mixed(86, 50, 47, K=5, C=3)
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 32, 2, 5, 0.002)
    out = []
    for use_graph, tuning in ((0, None), (1, None), (0, (2, 2))):
        with _ctx(lib, sc, use_graph=use_graph) as ctx:
            if tuning:
                ctx.set_tuning(*tuning)
            ctx.set_images(A0)
            ctx.iterate(2, 16, 2, 13)
            out.append((ctx.indirect(), ctx.normals(), ctx.depth()))
    for o in out[1:]:
        for x, y in zip(out[0], o):
            assert np.array_equal(x, y)


def test_shared_batch_matches_single_contexts(lib, oracle_mod):
    """A batch of light-shared objects (one persistent launch, per-object chunking and partial
    sums, batched zero and reduce) traces and solves the normals bit for bit as each object's
    own context, and a batched loop matches the oracle's light-shared loop per object."""
    spec = [(91, 24, 20, 4, 16, 1), (92, 17, 33, 8, 8, 2), (93, 30, 30, 6, 12, 2), (94, 9, 41, 5, 4, 1)]
    scs = [scenes.mixed(sd, H, W, K=K, C=3) for sd, H, W, K, _, _ in spec]
    A = [oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 32, 2, 3 + i, 0.002)
         for i, sc in enumerate(scs)]
    spp = [x[4] for x in spec]
    bounces = [x[5] for x in spec]
    ctxs = [_ctx(lib, sc) for sc in scs]
    try:
        for c, a in zip(ctxs, A):
            c.set_images(a)
        with lib.Batch(ctxs, use_graph=True) as b:
            b.iterate(1, spp, bounces, 41)
            st = b.stats()
            got = [(c.indirect(), c.normals()) for c in ctxs]
            b.iterate(1, spp, bounces, 41)
            got2 = [(c.normals(), c.depth()) for c in ctxs]
        assert st["walk_overflows"] == 0
        assert st["primary_segments"] == sum(sc.H * sc.W * s for sc, s in zip(scs, spp))
        for i, sc in enumerate(scs):
            with _ctx(lib, sc) as c:
                c.set_object(i)
                c.set_images(A[i])
                c.iterate(1, spp[i], bounces[i], 41)
                assert np.array_equal(got[i][0], c.indirect()), i
                assert np.array_equal(got[i][1], c.normals()), i
            hist = oracle_mod.irtps_run(A[i], sc.lights, sc.env, 2, spp[i], bounces[i], 41, obj=i, shared=True)
            err = oracle_mod.angular_error_deg(got2[i][0][..., :3].reshape(-1, 3), hist[2]["normals"].reshape(-1, 3))
            dabs = np.abs(got2[i][1] - hist[2]["depth"]) / np.ptp(hist[2]["depth"])
            assert err.mean() <= 0.05 and dabs.mean() <= 1e-4 and dabs.max() <= 1e-3, (i, err.mean(), dabs.max())
    finally:
        for c in ctxs:
            c.close()


def test_batch_rejects_mixed_sampling(lib):
    sc = scenes.mixed(87, 20, 20, K=4, C=3)
    with _ctx(lib, sc) as a, lib.Context(sc.H, sc.W, sc.lights, sc.env) as b:
        with pytest.raises(lib.IrtpsError) as e:
            lib.Batch([a, b])
        assert e.value.code == lib.IRTPS_EINVAL
