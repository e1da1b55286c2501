"""The whole IRT-PS loop in the oracle, on the 64x64 bowl (no GPU).

The paper reports (Table 1 and the discussion after it) that iterating the
reverted trace lowers height, albedo and normal error relative to classic PS.
On the concave bowl under a grey environment, where inter-reflection and the
environment make classic PS see a shallower, brighter surface, the oracle must
show the same trend; the convergence measure D_H must also shrink.
"""
import numpy as np

import scenes


def test_bowl_loop_improves_on_classic_ps(oracle_mod):
    sc = scenes.bowl_64()
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 256, 1, 1, 0.002)
    hist = oracle_mod.irtps_run(A0, sc.lights, sc.env, 3, 64, 1, 1)
    e = [(oracle_mod.height_error(sc.depth, h["depth"]), oracle_mod.albedo_error(sc.albedo, h["albedo"]),
          float(np.mean(oracle_mod.angular_error_deg(sc.normals, h["normals"])))) for h in hist]
    classic, last = e[0], e[-1]
    assert last[0] < 0.5 * classic[0]   # height
    assert last[1] < 0.5 * classic[1]   # albedo
    assert last[2] < classic[2]         # normal
    dh = [h["dH"][0] for h in hist[1:]]
    assert dh[-1] < dh[0]
    # classic PS on these images is biased: albedo overestimated by the extra light
    assert np.mean(hist[0]["albedo"]) > 0.7
