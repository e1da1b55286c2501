"""Pins of oracle parts that the other CPU tests leave open (no GPU).

Each expected value below comes from geometry, calculus or a hand-worked case,
never from the oracle itself:

* Environment lookup, azimuth (the known environment of Sec. IV): directions at
  texel centres return the texel exactly, a texel edge returns the mean of its two
  neighbours, the wrap across phi = 0 / 2 pi blends the last and first columns,
  and +y lies a quarter turn from +x.  A trace over a flat surface whose normal
  estimate is tilted, under a map L = a + b cos(phi), averages to an independent
  Gauss-Legendre integral of the interpolated map over the cosine lobe.
* Hit pixel (the pixel whose estimate a path reads at a hit): rays onto a tilted
  plane whose hit points are known in closed form, including points exactly
  halfway between vertices, which go to the lower index.
* Two-bounce transport (Sec. IV; the throughput product of the colour-extraction
  figure): in a 90-degree V-groove, the second-bounce increment of Lbar equals the
  nested view-factor integral of the groove (2D view factors of its facets; the
  inner factor integrated over the outer hit distribution by Gauss-Legendre)
  within 3 standard errors.
* D_H (the stopping rule of Sec. IV): a hand-worked pair of surfaces.
"""
import numpy as np

import scenes


# ---------------------------------------------------------------------------
# environment lookup, azimuth
# ---------------------------------------------------------------------------
def _dir(theta, phi):
    return np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])


def test_env_texel_centres_edges_and_wrap(oracle_mod):
    EH, EW = 4, 8
    env = (10.0 * np.arange(EH)[:, None] + np.arange(EW)[None, :] + 1.0)[None].astype(np.float32)
    m = env[0].astype(np.float64)
    dirs, want = [], []
    for r in range(EH):
        th = (r + 0.5) * np.pi / EH
        for c in range(EW):
            dirs.append(_dir(th, (c + 0.5) * 2 * np.pi / EW))    # texel centre: the texel itself
            want.append(m[r, c])
            dirs.append(_dir(th, c * 2 * np.pi / EW))            # left edge: mean with the column before
            want.append(0.5 * (m[r, c] + m[r, (c - 1) % EW]))
        # a quarter texel before phi = 2 pi: 3/4 of the last column, 1/4 of the first
        dirs.append(_dir(th, 2 * np.pi - 0.25 * 2 * np.pi / EW))
        want.append(0.75 * m[r, EW - 1] + 0.25 * m[r, 0])
        # the same angle reached from below zero (y < 0): atan2 wraps to [0, 2 pi)
        dirs.append(_dir(th, -0.25 * 2 * np.pi / EW))
        want.append(0.75 * m[r, EW - 1] + 0.25 * m[r, 0])
    # +y is a quarter turn from +x: column EW/4 - 1/2 (between columns 1 and 2 for EW = 8)
    dirs.append(np.array([0.0, 1.0, 0.0]))
    want.append(0.5 * (m[1, 1] + m[1, 2]) * 0.5 + 0.5 * (m[2, 1] + m[2, 2]) * 0.5)  # theta = pi/2: rows 1, 2
    # -x: half a turn, columns 3 and 4
    dirs.append(np.array([-1.0, 0.0, 0.0]))
    want.append(0.25 * (m[1, 3] + m[1, 4] + m[2, 3] + m[2, 4]))
    # near the pole theta -> 0 the rows clamp to row 0
    dirs.append(_dir(0.1 * np.pi / EH, (2 + 0.5) * 2 * np.pi / EW))
    want.append(m[0, 2])
    got = oracle_mod.env_lookup(env, np.array(dirs))
    assert np.abs(got - np.array(want)).max() < 1e-12


def _interp_phi(vals, phi):
    """The map's value along phi: linear between column centres (c + 1/2) 2 pi / EW, periodic."""
    EW = vals.size
    col = phi / (2 * np.pi) * EW - 0.5
    c0 = np.floor(col)
    f = col - c0
    a = vals[np.mod(c0, EW).astype(int)]
    b = vals[np.mod(c0 + 1, EW).astype(int)]
    return (1 - f) * a + f * b


def _tilted_lobe_expectation(vals, n, n_beta=2048, n_alpha=96):
    """E[L(w) 1{w_z > 0}] for w cosine-distributed about n (density (n.w)/pi), L = the map
    along phi; by the trapezoid rule in the azimuth beta about n (periodic) and
    Gauss-Legendre in the polar angle alpha up to the horizon w_z = 0."""
    n = n / np.linalg.norm(n)
    t1 = np.cross([0.0, 0.0, 1.0], n)
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    xg, wg = np.polynomial.legendre.leggauss(n_alpha)
    total = 0.0
    for beta in (np.arange(n_beta) + 0.5) * 2 * np.pi / n_beta:
        u = np.cos(beta) * t1 + np.sin(beta) * t2
        A, B = u[2], n[2]                     # w_z(alpha) = A sin(alpha) + B cos(alpha), B > 0
        top = np.pi / 2 if A >= 0 else min(np.pi / 2, np.arctan2(B, -A))
        al = 0.5 * top * (xg + 1.0)
        w = np.sin(al)[:, None] * u[None] + np.cos(al)[:, None] * n[None]
        phi = np.mod(np.arctan2(w[:, 1], w[:, 0]), 2 * np.pi)
        f = _interp_phi(vals, phi) * np.cos(al) * np.sin(al) / np.pi
        total += 0.5 * top * np.sum(wg * f) * (2 * np.pi / n_beta)
    return total


def test_env_azimuth_through_trace_tilted_lobe(oracle_mod):
    """Flat surface, zero albedo (a hit adds nothing and ends the path), normal estimate tilted
    35 deg toward azimuth 0.9 rad: rays below the surface hit it within the start cell and
    rays above escape, so Lbar = E[L(w) 1{w_z > 0}] over the tilted cosine lobe."""
    H = W = 24
    EH, EW = 4, 16
    a, b = 0.5, 0.4
    vals = a + b * np.cos((np.arange(EW) + 0.5) * 2 * np.pi / EW)
    env = np.broadcast_to(vals[None, None, :], (1, EH, EW)).astype(np.float32)
    tau, psi = np.radians(35.0), 0.9
    n = np.array([np.sin(tau) * np.cos(psi), np.sin(tau) * np.sin(psi), np.cos(tau)])
    depth = np.zeros((H, W), np.float32)
    normals = np.broadcast_to(n.astype(np.float32), (H, W, 3)).copy()
    albedo = np.zeros((1, H, W), np.float32)
    lights = np.asarray(scenes.ring_lights(1, 50.0), np.float32)
    ii, jj = np.meshgrid(np.arange(4, 20), np.arange(4, 20), indexing="ij")
    pix = (ii * W + jj).ravel().astype(np.int32)
    spp = 2048
    lbar, _, _ = oracle_mod.trace(depth, normals, albedo, lights, env, spp, 1, 31, 0, pixels=pix,
                                  shadow_rays=False, fp32=True)
    est = lbar[0, 0]                               # independent per-pixel estimates
    exact = _tilted_lobe_expectation(vals.astype(np.float32).astype(np.float64), n)
    coarse = _tilted_lobe_expectation(vals.astype(np.float32).astype(np.float64), n, 1024, 48)
    se = est.std(ddof=1) / np.sqrt(est.size)
    # the map is piecewise linear in phi (kinks at column centres): the rules converge as
    # 1/n^2, so halving both point counts bounds the fine rule's error by |fine - coarse| / 3
    assert abs(exact - coarse) < 0.25 * se
    assert abs(est.mean() - exact) < 4 * se + abs(exact - coarse), (est.mean(), exact, se)
    # the test has the power to see an azimuth slip of half a texel or a swapped atan2
    slip = _tilted_lobe_expectation(_interp_phi(vals, (np.arange(EW) + 1.0) * 2 * np.pi / EW), n, 512, 48)
    swap = a + b * (_tilted_lobe_expectation(np.sin((np.arange(EW) + 0.5) * 2 * np.pi / EW), n, 512, 48))
    assert abs(slip - exact) > 20 * se and abs(swap - exact) > 20 * se


# ---------------------------------------------------------------------------
# hit pixel
# ---------------------------------------------------------------------------
def _nearest(q, n):
    """Nearest of the vertices 0..n-1 to coordinate q, ties to the lower index."""
    return min(range(n), key=lambda v: (abs(q - v), v))


def test_hit_pixel_tilted_plane(oracle_mod):
    H, W = 12, 10
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    depth = (0.25 + jj / 64.0 - ii / 32.0).astype(np.float32)   # exact in float32

    def z(x, y):
        return 0.25 + x / 64.0 - y / 32.0

    # vertical rays: the hit point is the origin's (x, y) exactly, in both precisions
    xs = [0.0, 0.25, 0.5, 0.5 + 2.0 ** -20, 1.5, 2.5, 3.5, 3.5 - 2.0 ** -20, 4.75, 7.5, 8.5, 8.75, 9.0]
    ys = [0.0, 0.5, 1.5, 2.5 + 2.0 ** -20, 5.5, 6.25, 10.5, 10.75, 11.0]
    rays, want = [], []
    for x in xs:
        for y in ys:
            rays.append([x, y, 5.0, 0.0, 0.0, -1.0])
            want.append(_nearest(y, H) * W + _nearest(x, W))
    # oblique rays onto chosen points (away from ties; the float hit point carries rounding)
    rng = np.random.default_rng(5)
    for _ in range(300):
        x, y = rng.uniform(0.2, W - 1.2), rng.uniform(0.2, H - 1.2)
        if min(abs(x - np.floor(x) - 0.5), abs(y - np.floor(y) - 0.5)) < 1e-3:
            continue
        d = np.array([rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), -1.0])
        t = rng.uniform(0.5, 1.5)
        o = np.array([x, y, z(x, y)]) - t * d
        if not (0.0 <= o[0] <= W - 1 and 0.0 <= o[1] <= H - 1):
            continue  # paths start on the mesh (pixel vertices, hit points), never beside it
        rays.append([*o, *d])
        want.append(_nearest(y, H) * W + _nearest(x, W))
    rays = np.array(rays)
    for fp32 in (True, False):
        got = oracle_mod.hit_pixels(depth, rays, fp32=fp32)
        assert np.array_equal(got, np.array(want)), np.nonzero(got != np.array(want))
    # a ray that leaves the mesh upward has no hit pixel
    assert oracle_mod.hit_pixels(depth, np.array([[3.0, 3.0, 1.0, 0.1, 0.0, 1.0]]))[0] == -1


# ---------------------------------------------------------------------------
# two-bounce transport in a V-groove
# ---------------------------------------------------------------------------
def _groove_view_factors(a, Lf, n=200):
    """2D view factors of a 90-degree V-groove with facets of length Lf (lines along the groove,
    infinitely long): from a point at distance a from the bottom on one facet,
    F1 = P(the cosine-sampled ray meets the other facet) = (1 - a / sqrt(a^2 + Lf^2)) / 2, and
    P12 = P(it meets the other facet, and a cosine-sampled ray from that hit point meets the
    first facet) = int_0^Lf dF1/db (b) F1(b; from b) db, by Gauss-Legendre."""
    f1 = 0.5 * (1.0 - a / np.hypot(a, Lf))
    xg, wg = np.polynomial.legendre.leggauss(n)
    bb = 0.5 * Lf * (xg + 1.0)
    dens = 0.5 * a * bb / (a * a + bb * bb) ** 1.5
    back = 0.5 * (1.0 - bb / np.hypot(bb, Lf))
    p12 = 0.5 * Lf * np.sum(wg * dens * back)
    # the density integrates to F1 (a check on the quadrature)
    assert abs(0.5 * Lf * np.sum(wg * dens) - f1) < 1e-12
    return f1, p12


def _groove_case(oracle_mod, rho_a, rho_b):
    W, j0 = 65, 32                  # bottom vertex column; facets 32 columns wide
    H = 1025                        # long along the groove, so that it acts as an infinite one
    jj = np.arange(W)
    depth = np.broadcast_to((np.abs(jj - j0) / W).astype(np.float32), (H, W)).copy()
    nA = np.array([-1.0, 0.0, 1.0]) / np.sqrt(2.0)   # facet j > j0 (rising with x)
    nB = np.array([1.0, 0.0, 1.0]) / np.sqrt(2.0)    # facet j <= j0
    normals = np.where((jj > j0)[None, :, None], nA, nB).astype(np.float32)
    normals = np.broadcast_to(normals, (H, W, 3)).copy()
    albedo = np.broadcast_to(np.where(jj > j0, rho_a, rho_b).astype(np.float32), (1, H, W)).copy()
    l = np.array([[0.0, 0.6, 0.8]], np.float32)        # in the plane of the groove: V = 1 everywhere
    E = 1.0
    env = np.full((1, 4, 8), E, np.float32)
    jp = j0 + 16                                       # a = Lf / 2
    pix = (np.arange(384, 641, 4) * W + jp).astype(np.int32)
    spp = 4096
    l1, _, _ = oracle_mod.trace(depth, normals, albedo, l, env, spp, 1, 17, 0, pixels=pix)
    l2, _, _ = oracle_mod.trace(depth, normals, albedo, l, env, spp, 2, 17, 0, pixels=pix)
    inc = (l2 - l1)[0, 0]            # bounce 1 draws the same numbers in both: the bounce-2 term
    a, Lf = np.sqrt(2.0) * (jp - j0) / W, np.sqrt(2.0) * j0 / W
    f1, p12 = _groove_view_factors(a, Lf)
    cl = float(nA @ l[0].astype(np.float64))
    # hit on the other facet (throughput rho_b), then escape: rho_b E; or a second hit back on
    # the first facet: rho_b rho_a (n_A . l) V with V = 1
    want = rho_b * (E * (f1 - p12) + rho_a * cl * p12)
    # standard error of the per-pixel means (pixels are independent, equivalent estimates)
    se = inc.std(ddof=1) / np.sqrt(inc.size)
    return inc.mean(), want, se, (f1, p12, cl)


def test_bounce2_vgroove_matches_view_factor_integral(oracle_mod):
    got, want, se, _ = _groove_case(oracle_mod, 0.5, 0.5)
    assert abs(got - want) < 3 * se, (got, want, se)
    # an extra cosine in the throughput (E[cos] = 2/3) or a dropped albedo would be seen
    assert abs(want * 2 / 3 - want) > 6 * se and abs(want / 0.5 - want) > 6 * se


def test_bounce2_vgroove_albedo_of_each_hit(oracle_mod):
    """Different facet albedos: the throughput takes the first hit's albedo (rho_b), the
    second hit's direct term its own (rho_a)."""
    got, want, se, (f1, p12, cl) = _groove_case(oracle_mod, 0.5, 0.3)
    assert abs(got - want) < 3 * se, (got, want, se)
    wrong = 0.5 * (1.0 * (f1 - p12) + 0.3 * cl * p12)  # throughput from the origin's albedo instead
    assert abs(wrong - want) > 6 * se


# ---------------------------------------------------------------------------
# D_H
# ---------------------------------------------------------------------------
def test_dh_hand_worked(oracle_mod):
    h_old = np.array([[0.0, 1.0], [2.0, 3.0]])
    h_new = np.array([[0.0, 1.5], [2.0, 4.0]])
    dh, rms = oracle_mod.diff_norm(h_new, h_old)
    # max |change| = 1 at (1, 1); range of the NEW surface = 4 - 0 = 4; RMS = sqrt((0.25 + 1) / 4)
    assert dh == 0.25
    assert abs(rms - np.sqrt(1.25 / 4.0)) < 1e-15
    # a flat new surface has no range: D_H is 0 by convention, RMS still the change
    dh0, rms0 = oracle_mod.diff_norm(np.full((2, 2), 7.0), h_old)
    assert dh0 == 0.0 and abs(rms0 - np.sqrt(((7 - h_old) ** 2).mean())) < 1e-15
