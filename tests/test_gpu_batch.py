"""Batches: many objects of different sizes, light counts, sample counts and
bounce counts iterated with one launch per stage.

* Against the oracle loop, object by object (object index i in the Philox key).
* Against each object's own context: the first batched iteration traces and
  solves the normals bit for bit as the single-object path; the depth solve
  differs only by the team size of its reductions.
* A captured-and-replayed batch iteration gives the same bits as the enqueued one.
* The tuning knobs (trace grid, pyramid levels) change no result bit.
"""
import numpy as np
import pytest

import scenes
from stagewise import check_iteration, snapshot

pytestmark = pytest.mark.gpu

# (seed, H, W, K, spp, bounces): ragged sizes, every combination of the knobs that differ
SMALL = [(61, 24, 20, 4, 16, 1), (62, 17, 33, 8, 8, 2), (63, 30, 30, 6, 12, 2), (64, 9, 41, 5, 4, 1)]


def _scenes(spec):
    return [scenes.mixed(s, H, W, K=K, C=3) for s, H, W, K, _, _ in spec]


def _images(oracle_mod, scs, seed=5):
    return [oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 32, 2, seed + i, 0.002)
            for i, sc in enumerate(scs)]


def test_batch_matches_oracle(lib, oracle_mod):
    scs = _scenes(SMALL)
    A = _images(oracle_mod, scs)
    spp = [s[4] for s in SMALL]
    bounces = [s[5] for s in SMALL]
    seed, n_iter = 17, 2
    ctxs = [lib.Context(sc.H, sc.W, sc.lights, sc.env) for sc in scs]
    try:
        for c, a in zip(ctxs, A):
            c.set_images(a)
        with lib.Batch(ctxs) as b:
            for t in range(n_iter):  # each object's iteration t checked stage by stage from its own state
                before = [snapshot(c) for c in ctxs]
                dh = b.iterate(1, spp, bounces, seed)
                st = b.stats()
                assert st["walk_overflows"] == 0 and st["cg_rel_residual"] <= 1e-9
                assert st["primary_segments"] == sum(sc.H * sc.W * sc.K * s for sc, s in zip(scs, spp))
                for i, (sc, c, a) in enumerate(zip(scs, ctxs, A)):
                    dh_o = check_iteration(oracle_mod, a, sc.lights, sc.env, before[i], snapshot(c), c.indirect(),
                                           spp[i], bounces[i], seed, t, obj=i)
                    assert abs(dh[i] - dh_o) <= 1e-9 + 1e-6 * dh_o, (i, t, dh[i], dh_o)
        # secondary: the free-running loops from the same images
        for i, (sc, c, a) in enumerate(zip(scs, ctxs, A)):
            hist = oracle_mod.irtps_run(a, sc.lights, sc.env, n_iter, spp[i], bounces[i], seed, obj=i)
            h = hist[-1]
            n, d = c.normals(), c.depth()
            err = oracle_mod.angular_error_deg(n[..., :3].reshape(-1, 3), h["normals"].reshape(-1, 3))
            dabs = np.abs(d - h["depth"]) / np.ptp(h["depth"])
            assert err.mean() <= 0.05, (i, err.mean())
            assert dabs.mean() <= 1e-4 and dabs.max() <= 1e-3, (i, dabs.mean(), dabs.max())
    finally:
        for c in ctxs:
            c.close()


def _single(lib, sc, a, obj, n_iter, spp, bounces, seed):
    with lib.Context(sc.H, sc.W, sc.lights, sc.env) as c:
        c.set_object(obj)
        c.set_images(a)
        c.iterate(n_iter, spp, bounces, seed)
        return c.indirect(), c.normals(), c.albedo(), c.depth(), c.valid()


def test_batch_matches_single_contexts(lib, oracle_mod):
    spec = SMALL + [(65, 64, 48, 12, 8, 2)]
    scs = _scenes(spec)
    A = _images(oracle_mod, scs, 9)
    spp = [s[4] for s in spec]
    bounces = [s[5] for s in spec]
    seed = 23
    ctxs = [lib.Context(sc.H, sc.W, sc.lights, sc.env) for sc in scs]
    try:
        for c, a in zip(ctxs, A):
            c.set_images(a)
        with lib.Batch(ctxs) as b:
            b.iterate(1, spp, bounces, seed)
            got1 = [(c.indirect(), c.normals(), c.albedo(), c.depth(), c.valid()) for c in ctxs]
            b.iterate(1, spp, bounces, seed)  # the iteration index continues per object
            got2 = [(c.normals(), c.depth()) for c in ctxs]
        for i, sc in enumerate(scs):
            lb, n, al, d, v = _single(lib, sc, A[i], i, 1, spp[i], bounces[i], seed)
            assert np.array_equal(got1[i][0], lb), i  # trace: bit-identical
            assert np.array_equal(got1[i][1], n), i   # PS: bit-identical
            assert np.array_equal(got1[i][2], al), i
            assert np.array_equal(got1[i][4], v), i
            assert np.abs(got1[i][3] - d).max() <= 1e-6 * np.ptp(d), i
            _, n2, _, d2, _ = _single(lib, sc, A[i], i, 2, spp[i], bounces[i], seed)
            err = oracle_mod.angular_error_deg(got2[i][0][..., :3].reshape(-1, 3), n2[..., :3].reshape(-1, 3))
            assert err.mean() <= 0.05, (i, err.mean())
            assert np.abs(got2[i][1] - d2).max() <= 1e-4 * np.ptp(d2), i
    finally:
        for c in ctxs:
            c.close()


def test_batch_graph_replay_and_tuning_match(lib, oracle_mod):
    scs = _scenes(SMALL)
    A = _images(oracle_mod, scs, 13)
    spp = [s[4] for s in SMALL]
    bounces = [s[5] for s in SMALL]
    runs = []
    for use_graph, tuning in ((False, None), (True, None), (False, (1, 2)), (True, (2, 1))):
        ctxs = [lib.Context(sc.H, sc.W, sc.lights, sc.env) for sc in scs]
        try:
            for c, a in zip(ctxs, A):
                c.set_images(a)
            with lib.Batch(ctxs, use_graph=use_graph) as b:
                if tuning:
                    b.set_tuning(*tuning)
                    assert b.tuning() == tuning
                b.iterate(2, spp, bounces, 31)
                b.iterate(1, spp, bounces, 31)
                runs.append([(c.indirect(), c.normals(), c.depth()) for c in ctxs])
        finally:
            for c in ctxs:
                c.close()
    for r in runs[1:]:
        for x, y in zip(runs[0], r):
            for u, v in zip(x, y):
                assert np.array_equal(u, v)


def test_single_tuning_and_autotune_keep_results(lib, oracle_mod):
    sc = scenes.mixed(71, 96, 80, K=8, C=3)
    res = []
    with lib.Context(sc.H, sc.W, sc.lights, sc.env) as c:
        c.set_state(sc.depth, sc.normals, sc.albedo)
        for bps, cut in ((0, 0), (1, 0), (2, 3), (3, 1)):
            c.set_tuning(bps, cut)
            c.trace(16, 2, 3, 0)
            res.append(c.indirect())
        ms = c.autotune(4, 2, 3)
        assert ms > 0.0
        bps, cut = c.tuning()
        assert bps >= 1 and cut >= 0
        c.trace(16, 2, 3, 0)
        res.append(c.indirect())
    for r in res[1:]:
        assert np.array_equal(res[0], r)


def test_batch_autotune_and_errors(lib, oracle_mod):
    scs = _scenes(SMALL[:2])
    A = _images(oracle_mod, scs, 3)
    ctxs = [lib.Context(sc.H, sc.W, sc.lights, sc.env) for sc in scs]
    mono = scenes.mixed(80, 20, 20, K=4, C=1)
    try:
        with lib.Batch(ctxs) as b:
            with pytest.raises(lib.IrtpsError) as e:  # images not set yet
                b.iterate(1, [4, 4], [1, 1], 1)
            assert e.value.code == lib.IRTPS_ENOTREADY
            for c, a in zip(ctxs, A):
                c.set_images(a)
            with pytest.raises(lib.IrtpsError) as e:
                b.iterate(1, [4, 0], [1, 1], 1)
            assert e.value.code == lib.IRTPS_EINVAL
            with pytest.raises(lib.IrtpsError) as e:
                b.iterate(1, [4, 4], [1, 4], 1)
            assert e.value.code == lib.IRTPS_EINVAL
            ms = b.autotune([2, 2], [1, 2], 5)
            assert ms > 0.0
            b.iterate(1, [4, 4], [1, 2], 5)
            assert b.stats()["walk_overflows"] == 0
        with lib.Context(mono.H, mono.W, mono.lights, mono.env) as m:
            with pytest.raises(lib.IrtpsError) as e:  # channel counts differ
                lib.Batch(ctxs + [m])
            assert e.value.code == lib.IRTPS_EINVAL
        with pytest.raises(lib.IrtpsError):  # the same context twice
            lib.Batch([ctxs[0], ctxs[0]])
    finally:
        for c in ctxs:
            c.close()


def test_batch_set_images_matches_single(lib, oracle_mod):
    """Batched iteration 0 (classic PS and integration of every object) against each
    object's irtps_set_images: normals bit-identical, depth within the solver's tolerance;
    then a batched iteration over it matches the oracle loop."""
    scs = _scenes(SMALL)
    A = _images(oracle_mod, scs, 19)
    ctxs = [lib.Context(sc.H, sc.W, sc.lights, sc.env) for sc in scs]
    try:
        with lib.Batch(ctxs) as b:
            b.set_images(A)
            st = b.stats()
            assert st["cg_rel_residual"] <= 1e-9
            got = [(c.normals(), c.depth(), c.valid()) for c in ctxs]
            spp = [s[4] for s in SMALL]
            bounces = [s[5] for s in SMALL]
            b.iterate(1, spp, bounces, 3)
            after = [(c.normals(), c.depth()) for c in ctxs]
        for i, (sc, a) in enumerate(zip(scs, A)):
            with lib.Context(sc.H, sc.W, sc.lights, sc.env) as c:
                c.set_images(a)
                n, d, v = c.normals(), c.depth(), c.valid()
            assert np.array_equal(got[i][0], n), i
            assert np.array_equal(got[i][2], v), i
            assert np.abs(got[i][1] - d).max() <= 1e-6 * np.ptp(d), i
            hist = oracle_mod.irtps_run(a, sc.lights, sc.env, 1, spp[i], bounces[i], 3, obj=i)
            err = oracle_mod.angular_error_deg(after[i][0][..., :3].reshape(-1, 3), hist[1]["normals"].reshape(-1, 3))
            dabs = np.abs(after[i][1] - hist[1]["depth"]) / np.ptp(hist[1]["depth"])
            assert err.mean() <= 0.05 and dabs.mean() <= 1e-4 and dabs.max() <= 1e-3, (i, err.mean(), dabs.max())
    finally:
        for c in ctxs:
            c.close()


def test_batch_robust_integration(lib, oracle_mod):
    """Objects with robust integration (Huber IRLS, the same number of reweighting steps,
    their own thresholds) in one batch: iteration 0 gives each object's own normals bit for
    bit and its surface within the solver's tolerance; a batched iteration matches the
    oracle's robust loop."""
    scs = _scenes(SMALL)
    A = _images(oracle_mod, scs, 23)
    deltas = [0.05, 0.08, 0.05, 0.03]
    ctxs = []
    for sc, dl in zip(scs, deltas):
        opt = lib.irtps_default_options()
        opt.irls_iters = 2
        opt.irls_delta = dl
        ctxs.append(lib.Context(sc.H, sc.W, sc.lights, sc.env, opt))
    spp = [s[4] for s in SMALL]
    bounces = [s[5] for s in SMALL]
    try:
        with lib.Batch(ctxs) as b:
            b.set_images(A)
            assert b.stats()["cg_rel_residual"] <= 1e-9
            got0 = [(c.normals(), c.depth()) for c in ctxs]
            before = [snapshot(c) for c in ctxs]
            b.iterate(1, spp, bounces, 7)
            assert b.stats()["cg_rel_residual"] <= 1e-9
            got1 = [(c.normals(), c.depth()) for c in ctxs]
            for i, (sc, c, a, dl) in enumerate(zip(scs, ctxs, A, deltas)):
                check_iteration(oracle_mod, a, sc.lights, sc.env, before[i], snapshot(c), c.indirect(), spp[i],
                                bounces[i], 7, 0, obj=i, irls=(dl, 2))
        for i, (sc, a, dl) in enumerate(zip(scs, A, deltas)):
            opt = lib.irtps_default_options()
            opt.irls_iters = 2
            opt.irls_delta = dl
            with lib.Context(sc.H, sc.W, sc.lights, sc.env, opt) as c:
                c.set_images(a)
                assert np.array_equal(got0[i][0], c.normals()), i
                d = c.depth()
                assert np.abs(got0[i][1] - d).max() <= 1e-5 * np.ptp(d), i
            hist = oracle_mod.irtps_run(a, sc.lights, sc.env, 1, spp[i], bounces[i], 7, obj=i, irls_iters=2,
                                        irls_delta=dl)
            err = oracle_mod.angular_error_deg(got1[i][0][..., :3].reshape(-1, 3), hist[1]["normals"].reshape(-1, 3))
            dabs = np.abs(got1[i][1] - hist[1]["depth"]) / np.ptp(hist[1]["depth"])
            assert err.mean() <= 0.05 and dabs.mean() <= 1e-4 and dabs.max() <= 1e-3, (i, err.mean(), dabs.max())
        mixed = [lib.Context(scs[0].H, scs[0].W, scs[0].lights, scs[0].env)]
        with pytest.raises(lib.IrtpsError):  # reweighting steps must agree across the batch
            lib.Batch([ctxs[0], mixed[0]])
        mixed[0].close()
    finally:
        for c in ctxs:
            c.close()


def test_batch_early_escape_keeps_every_bit(lib, oracle_mod):
    """Batched horizon bounds (one launch over all objects) let rising primary rays
    skip their march; every object's Lbar and normals stay those of the plain batch."""
    spec = SMALL + [(66, 64, 48, 12, 8, 2)]
    scs = _scenes(spec)
    A = _images(oracle_mod, scs, 13)
    spp = [s[4] for s in spec]
    bounces = [s[5] for s in spec]
    out, visits = [], []
    for early in (0, 1):
        opt = lib.irtps_default_options()
        opt.early_escape = early
        ctxs = [lib.Context(sc.H, sc.W, sc.lights, sc.env, opt) for sc in scs]
        try:
            for c, a in zip(ctxs, A):
                c.set_images(a)
            with lib.Batch(ctxs) as b:
                b.iterate(1, spp, bounces, 29)
                visits.append(b.stats()["node_visits"])
                out.append([(c.indirect(), c.normals()) for c in ctxs])
        finally:
            for c in ctxs:
                c.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert visits[1] < visits[0]
