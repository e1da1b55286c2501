"""IRT-PS oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 CPU statement of what the IRT-PS hot path computes, written
from the paper (Khadka, Remagnino, Argyriou, "Object 3D Reconstruction based on
Photometric Stereo and Inverted Rendering", arXiv:1811.02357).  Only `tests/`,
`__graft_entry__.smoke()` and the benchmark's CPU-baseline / reference leg may
import it.  The CUDA library never does, and the two share no code: the trace
lives in `irtps_oracle.cpp` (plain C++, FP64 sums, geometry templated so that a
float instantiation takes integer decisions in the kernel's precision), the
photometric-stereo and integration steps live here in numpy/scipy.

Functions and the passages they follow:

* `pinv_lights`      — Eq. 4 (least squares with the transpose of L).
* `correct_images`   — the image correction of stage 5, A - E, read as
                       I = A0 - rho_t * Lbar_t (subtract from the original images).
* `valid_rows`       — shadow / saturation mask (the paper is silent; thresholds
                       tau_lo < I < tau_hi on the channel mean, decided in FP32).
* `ps_solve`         — Eq. 3-4 per pixel, masked rows re-solved by 3x3 normal
                       equations; n = direction, rho = length (text after Eq. 4).
* `poisson_solve`    — integration of the normals into H_t (stage 1, "integrating
                       over the obtained normals"): least-squares surface with
                       trapezoidal edge gradients, mean zero, solved exactly by
                       the cosine transform that diagonalises the Neumann Laplacian.
* `trace`            — Eq. 5-7 Monte-Carlo estimate of the indirect light with
                       cosine-weighted sampling, the reverted trace of Sec. IV,
                       bounce throughput c1*c2*c3 (figure on environment colour
                       extraction).
* `render`           — stage 0 synthetic input images (direct + traced indirect +
                       Gaussian noise).
* `hole_mask`, `interpolate_holes` — the single-sample variant of Sec. IV: pixels
                       whose samples saw no surface point get no environment value
                       and are filled by a non-uniform (pull-push) interpolation.
* `irtps_run`        — the loop of Sec. IV: PS, integrate, trace, subtract, repeat;
                       D_H = H_{t+1} - H_t reported per iteration.
* `height_error`, `albedo_error`, `normal_error` — the evaluation formulas of Sec. V.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
from scipy.fft import dctn, idctn

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "irtps_oracle.cpp")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

TAU_LO = 0.02
TAU_HI = 0.98
COND_MAX = 1e8
NZ_MIN = 0.05
FORWARD_ITER = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the C++ trace oracle (g++, FP contraction off) into oracle/_build."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, u32, u64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_cosine_dirs.argtypes = [i32, P, P, P, i32, P]
            lib.oracle_onb.argtypes = [i32, P, P, P]
            lib.oracle_sincos_turn.argtypes = [i32, P, i32, P, P]
            lib.oracle_tri_hit.argtypes = [i32, P, i32, P]
            lib.oracle_intersect.argtypes = [i32, i32, P, i32, P, i32, i32, P, P]
            lib.oracle_env_lookup.argtypes = [P, i32, i32, i32, i32, P, P]
            lib.oracle_hit_pixels.argtypes = [i32, i32, P, i32, P, i32, P]
            lib.oracle_trace.argtypes = [i32, i32, i32, i32, P, P, P, P, P, i32, i32, P, i32, i32, i32,
                                         u64, u32, u32, u32, i32, i32, i32, P, P, P]
            lib.oracle_trace.restype = i32
            lib.oracle_trace_shared.argtypes = [i32, i32, i32, i32, P, P, P, P, P, i32, i32, P, i32, i32, i32,
                                         u64, u32, u32, u32, i32, i32, i32, P, P, P]
            lib.oracle_trace_shared.restype = i32
            lib.oracle_pixel_visibility.argtypes = [i32, i32, i32, P, P, P, i32, P]
            lib.oracle_pixel_visibility.restype = i32
            lib.oracle_noise.argtypes = [i32, i32, i32, i32, u64, u32, P]
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------
# Random numbers and sampling
# ----------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11) of one 4-word counter and 2-word key."""
    lib = _load()
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def cosine_dirs(normals, x0, x1, fp32=False):
    """Cosine-weighted directions about each normal (Malley's method, Duff basis)."""
    lib = _load()
    n = _c(normals, np.float64).reshape(-1, 3)
    a = _c(x0, np.uint32)
    b = _c(x1, np.uint32)
    out = np.zeros((n.shape[0], 3))
    lib.oracle_cosine_dirs(n.shape[0], _ptr(n), _ptr(a), _ptr(b), int(fp32), _ptr(out))
    return out


def onb(normals):
    lib = _load()
    n = _c(normals, np.float64).reshape(-1, 3)
    b1 = np.zeros_like(n)
    b2 = np.zeros_like(n)
    lib.oracle_onb(n.shape[0], _ptr(n), _ptr(b1), _ptr(b2))
    return b1, b2


def sincos_turn(m, fp32=True):
    """cos(2 pi u), sin(2 pi u) for u = m / 2^24."""
    lib = _load()
    mm = _c(m, np.uint32)
    c = np.zeros(mm.size)
    s = np.zeros(mm.size)
    lib.oracle_sincos_turn(mm.size, _ptr(mm), int(fp32), _ptr(c), _ptr(s))
    return c, s


def tri_hit(rows, fp32=False):
    """Moeller-Trumbore on rows (o, d, v0, v1, v2); t or NaN."""
    lib = _load()
    r = _c(rows, np.float64).reshape(-1, 15)
    out = np.zeros(r.shape[0])
    lib.oracle_tri_hit(r.shape[0], _ptr(r), int(fp32), _ptr(out))
    return out


def intersect(depth, rays, fp32=False, brute=False):
    """Closest hit of grid-coordinate rays (o, d) with the meshed heightfield."""
    lib = _load()
    d = _c(depth, np.float32)
    H, W = d.shape
    r = _c(rays, np.float64).reshape(-1, 6)
    t = np.zeros(r.shape[0])
    tri = np.zeros(r.shape[0], np.int64)
    lib.oracle_intersect(H, W, _ptr(d), r.shape[0], _ptr(r), int(fp32), int(brute), _ptr(t), _ptr(tri))
    return t, tri


def hit_pixels(depth, rays, fp32=True):
    """Pixel index the trace shades at each ray's closest hit (nearest mesh vertex in x-y,
    ties to the lower index), or -1 for an escaping ray; rays (n, 6) in grid coordinates."""
    lib = _load()
    d = _c(depth, np.float32)
    H, W = d.shape
    r = _c(rays, np.float64).reshape(-1, 6)
    out = np.zeros(r.shape[0], np.int64)
    lib.oracle_hit_pixels(H, W, _ptr(d), r.shape[0], _ptr(r), int(fp32), _ptr(out))
    return out


def env_lookup(env, dirs, c=0):
    lib = _load()
    e = _c(env, np.float32)
    _, EH, EW = e.shape
    d = _c(dirs, np.float64).reshape(-1, 3)
    out = np.zeros(d.shape[0])
    lib.oracle_env_lookup(_ptr(e), EH, EW, c, d.shape[0], _ptr(d), _ptr(out))
    return out


# ----------------------------------------------------------------------------
# Trace and forward render
# ----------------------------------------------------------------------------
def pack_normals(normals, albedo):
    """(H, W, 3) normals and (C, H, W) albedo -> (H*W, 4) float32 (nx, ny, nz, mean albedo)."""
    n = np.asarray(normals, np.float32).reshape(-1, 3)
    a = np.asarray(albedo, np.float32)
    out = np.empty((n.shape[0], 4), np.float32)
    out[:, :3] = n
    out[:, 3] = a.reshape(a.shape[0], -1).mean(axis=0)
    return out


def trace(depth, normals, albedo, lights, env, spp, bounces, seed, iteration, *, pixels=None,
          stream=0, obj=0, shadow_rays=True, fp32=True, threads=0, records=False, shared=False):
    """Mean incident radiance Lbar (K, C, n_pix) of the reverted Monte-Carlo trace.

    depth (H, W), normals (H, W, 3), albedo (C, H, W) are the current estimate,
    rounded to float32 as the GPU stores them.  fp32=True decides hits in single
    precision (the kernel's); fp32=False in double.  Returns (lbar, records, counts):
    records (n_pix, K, spp, bounces, 2) int32 {hit pixel | -1 escape | -2 not reached,
    shadow visibility 1/0 | -1 not cast} when requested; counts = (primary, segments).

    shared=True: light-shared sampling, one path per (pixel, sample) for all K lights
    (directions drawn with light field 0); records then (n_pix, spp, bounces, 1 + K)
    {hit pixel | -1 | -2, V_0 .. V_{K-1}}.
    """
    lib = _load()
    d = _c(depth, np.float32)
    H, W = d.shape
    a = _c(albedo, np.float32)
    C = a.shape[0]
    n4 = pack_normals(normals, a)
    l = _c(lights, np.float32).reshape(-1, 3)
    K = l.shape[0]
    e = _c(env, np.float32)
    _, EH, EW = e.shape
    pix = None if pixels is None else _c(pixels, np.int32)
    n_pix = H * W if pix is None else pix.size
    out = np.zeros((K, C, n_pix))
    if shared:
        rec = np.zeros((n_pix, spp, bounces, 1 + K), np.int32) if records else None
    else:
        rec = np.zeros((n_pix, K, spp, bounces, 2), np.int32) if records else None
    counts = np.zeros(2, np.uint64)
    fn = lib.oracle_trace_shared if shared else lib.oracle_trace
    rc = fn(H, W, C, K, _ptr(d), _ptr(n4), _ptr(a), _ptr(l), _ptr(e), EH, EW, _ptr(pix),
                          n_pix, spp, bounces, int(seed), obj, int(iteration) & 0xFFFFFFFF, stream,
                          int(shadow_rays), int(fp32), int(threads), _ptr(out), _ptr(rec), _ptr(counts))
    if rc != 0:
        raise ValueError("oracle_trace: invalid arguments")
    return out, rec, (int(counts[0]), int(counts[1]))


def pixel_visibility(depth, normals, lights, fp32=True):
    """V_k(p) of each pixel's own vertex: (K, H, W) int32, 1/0, -1 when n.l <= 0."""
    lib = _load()
    d = _c(depth, np.float32)
    H, W = d.shape
    n4 = pack_normals(normals, np.ones((1, H, W), np.float32))
    l = _c(lights, np.float32).reshape(-1, 3)
    out = np.zeros((l.shape[0], H, W), np.int32)
    rc = lib.oracle_pixel_visibility(H, W, l.shape[0], _ptr(d), _ptr(n4), _ptr(l), int(fp32), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_pixel_visibility: invalid arguments")
    return out


def noise(H, W, C, K, seed, obj=0):
    """Standard normal deviates (K, C, H, W) of the image noise (Box-Muller on Philox, stream 2)."""
    lib = _load()
    out = np.zeros((K, C, H, W))
    lib.oracle_noise(H, W, C, K, int(seed), obj, _ptr(out))
    return out


def render(depth, normals, albedo, lights, env, spp, bounces, seed, sigma, *, shadow_rays=True,
           fp32=True, threads=0, indirect=True):
    """Stage-0 input images A0 (K, C, H, W) float32 of a ground-truth scene:
    A0 = rho * max(0, n.l_k) * V_k + rho * Lbar_gt + sigma * N(0, 1), with Lbar_gt
    traced on the ground truth with stream 1 and iteration 0xFFFFFFFF
    (indirect=False: the direct term and the noise only)."""
    d = np.asarray(depth, np.float32)
    H, W = d.shape
    a = np.asarray(albedo, np.float32)
    C = a.shape[0]
    n = np.asarray(normals, np.float32)
    l = np.asarray(lights, np.float32).reshape(-1, 3)
    K = l.shape[0]
    if indirect:
        lbar, _, _ = trace(d, n, a, l, env, spp, bounces, seed, FORWARD_ITER, stream=1,
                           shadow_rays=shadow_rays, fp32=fp32, threads=threads)
    else:
        lbar = np.zeros((K, C, H * W))
    vis = pixel_visibility(d, n, l, fp32=fp32) if shadow_rays else None
    n64 = n.reshape(-1, 3).astype(np.float64)
    cos = np.maximum(0.0, n64 @ l.astype(np.float64).T).T  # (K, P)
    if vis is not None:
        v = vis.reshape(K, -1)
        cos = np.where(v == 1, cos, 0.0)
    a64 = a.reshape(C, -1).astype(np.float64)
    direct = cos[:, None, :] * a64[None, :, :]
    indirect = a64[None, :, :] * lbar
    z = noise(H, W, C, K, seed).reshape(K, C, -1)
    return (direct + indirect + sigma * z).reshape(K, C, H, W).astype(np.float32)


# ----------------------------------------------------------------------------
# Single-sample holes and their interpolation (Sec. IV, environment colour images)
# ----------------------------------------------------------------------------
def hole_mask(records):
    """Holes of a per-light trace: (K, n_pix) bool, True where every sample of
    (pixel, light) left the surface at its first segment, so that the pixel saw no
    surface point and its environment image has no value there (Sec. IV: with a
    single sample some pixels get none).  records as returned by `trace`:
    (n_pix, K, spp, bounces, 2), field 0 of the first bounce = -1 on escape."""
    r = np.asarray(records)
    return np.all(r[:, :, :, 0, 0] == -1, axis=2).T


def pyramid_sizes(H, W):
    """Level sizes of the fill pyramid: halved (rounded up) until 1 x 1."""
    sizes = [(H, W)]
    while sizes[-1] != (1, 1):
        h, w = sizes[-1]
        sizes.append(((h + 1) // 2, (w + 1) // 2))
    return sizes


def _upsample_taps(n_fine, n_coarse):
    """Coarse neighbours and weights of each fine index for 2x linear upsampling of
    cell-centred samples: fine centre i sits at coarse coordinate i/2 - 1/4, so an
    even i takes (i/2 - 1, i/2) with weights (1/4, 3/4), an odd i takes
    ((i-1)/2, (i+1)/2) with (3/4, 1/4); indices clamp to the border."""
    i = np.arange(n_fine)
    lo = np.where(i % 2 == 0, i // 2 - 1, (i - 1) // 2)
    hi = lo + 1
    w_lo = np.where(i % 2 == 0, 0.25, 0.75)
    return np.clip(lo, 0, n_coarse - 1), np.clip(hi, 0, n_coarse - 1), w_lo, 1.0 - w_lo


def interpolate_holes(values, known):
    """Non-uniform interpolation of the missing pixels of environment images (the
    paper names a non-uniform interpolation without giving it; this is the pull-push
    form of multiscale normalised convolution).

    values (K, C, H, W), known (K, H, W) bool.  Pull: level l+1 holds, per coarse
    pixel, the sum S of its (up to four) children's confidences and the
    confidence-weighted mean of their values; its confidence is min(S, 1), with
    confidence 1 at known and 0 at missing pixels of level 0.  Push, from the 1 x 1
    level down: a pixel's value becomes w v + (1 - w) u, w its confidence and u the
    2x linear upsampling of the finished coarser level.  Known pixels keep their
    value; an image with no known pixel stays as it is.  FP64; returns a copy."""
    v0 = np.asarray(values, np.float64)
    w0 = np.asarray(known, bool).astype(np.float64)
    K, C, H, W = v0.shape
    sizes = pyramid_sizes(H, W)
    V, Wt = [v0], [w0]
    for (h, w), (h2, w2) in zip(sizes[:-1], sizes[1:]):
        wp = np.zeros((K, 2 * h2, 2 * w2))
        vp = np.zeros((K, C, 2 * h2, 2 * w2))
        wp[:, :h, :w] = Wt[-1]
        vp[:, :, :h, :w] = V[-1] * Wt[-1][:, None]
        s_w = wp[:, 0::2, 0::2] + wp[:, 1::2, 0::2] + wp[:, 0::2, 1::2] + wp[:, 1::2, 1::2]
        s_v = vp[:, :, 0::2, 0::2] + vp[:, :, 1::2, 0::2] + vp[:, :, 0::2, 1::2] + vp[:, :, 1::2, 1::2]
        has = s_w > 0
        V.append(np.where(has[:, None], s_v / np.where(has, s_w, 1.0)[:, None], 0.0))
        Wt.append(np.minimum(s_w, 1.0))
    out = V[-1]
    for lvl in range(len(sizes) - 2, -1, -1):
        h, w = sizes[lvl]
        h2, w2 = sizes[lvl + 1]
        y0, y1, a0, a1 = _upsample_taps(h, h2)
        x0, x1, b0, b1 = _upsample_taps(w, w2)
        u = (a0[:, None] * (b0[None, :] * out[:, :, y0][:, :, :, x0] + b1[None, :] * out[:, :, y0][:, :, :, x1]) +
             a1[:, None] * (b0[None, :] * out[:, :, y1][:, :, :, x0] + b1[None, :] * out[:, :, y1][:, :, :, x1]))
        wl = Wt[lvl][:, None]
        out = wl * V[lvl] + (1.0 - wl) * u
    none = Wt[-1][:, 0, 0] == 0  # images with no known pixel
    out[none] = v0[none]
    return out


# ----------------------------------------------------------------------------
# Photometric stereo (Eq. 3-4)
# ----------------------------------------------------------------------------
def pinv_lights(lights):
    """(L^T L)^{-1} L^T of the K x 3 illumination matrix (Eq. 4)."""
    L = np.asarray(lights, np.float64).reshape(-1, 3)
    return np.linalg.inv(L.T @ L) @ L.T


def correct_images(A0, rho, lbar):
    """I = A0 - rho_t * Lbar_t in FP64; shapes (K, C, P), (C, P), (K, C, P)."""
    return np.asarray(A0, np.float64) - np.asarray(rho, np.float64)[None] * np.asarray(lbar, np.float64)


def valid_rows(A0, rho, lbar, tau_lo=TAU_LO, tau_hi=TAU_HI):
    """Row k of pixel p is kept iff tau_lo < mean_c I(p,k,c) < tau_hi.

    The mask is an integer decision taken from floating point, so it is decided in
    FP32 with every operation rounded on its own: I = A0 - (rho * Lbar), channel mean
    ((I0 + I1) + I2) / 3.  Returns (K, P) bool."""
    f = np.float32
    A = np.asarray(A0, f)
    r = np.asarray(rho, f)
    lb = np.asarray(lbar, f)
    I = A - (r[None] * lb)
    C = I.shape[1]
    if C == 1:
        chat = I[:, 0]
    else:
        acc = I[:, 0]
        for c in range(1, C):
            acc = acc + I[:, c]
        chat = acc / f(C)
    return (chat > f(tau_lo)) & (chat < f(tau_hi))


def ps_solve(I, valid, lights, cond_max=COND_MAX):
    """Per-pixel Lambertian PS.  I (K, C, P) FP64, valid (K, P).

    All rows valid: G_c = pinv(L) I_c (Eq. 4).  Otherwise the FP64 normal equations
    (L_v^T L_v) G_c = L_v^T I_v,c over the valid rows; fewer than 3 rows or a 1-norm
    condition number above cond_max marks the pixel invalid.  n = normalize(sum_c G_c),
    rho_c = |G_c|; invalid pixels get n = (0, 0, 1), rho = 0.
    Returns n (P, 3), rho (C, P), ok (P,) bool."""
    I = np.asarray(I, np.float64)
    K, C, P = I.shape
    L = np.asarray(lights, np.float64).reshape(-1, 3)
    G = np.einsum("ak,kcp->acp", pinv_lights(L), I)  # (3, C, P)
    full = valid.all(axis=0)
    ok = full.copy()
    for p in np.nonzero(~full)[0]:
        v = valid[:, p]
        if v.sum() < 3:
            G[:, :, p] = 0.0
            continue
        Lv = L[v]
        M = Lv.T @ Lv
        if not np.isfinite(np.linalg.cond(M, 1)) or np.linalg.cond(M, 1) > cond_max:
            G[:, :, p] = 0.0
            continue
        G[:, :, p] = np.linalg.solve(M, Lv.T @ I[v, :, p])
        ok[p] = True
    s = G.sum(axis=1)  # (3, P)
    norm = np.sqrt((s * s).sum(axis=0))
    ok &= np.isfinite(norm) & (norm > 0)
    n = np.zeros((P, 3))
    n[:, 2] = 1.0
    safe = np.where(ok, norm, 1.0)
    n[ok] = (s / safe).T[ok]
    rho = np.sqrt((G * G).sum(axis=0))  # (C, P)
    rho[:, ~ok] = 0.0
    return n, rho, ok


# ----------------------------------------------------------------------------
# Integration (normals -> depth)
# ----------------------------------------------------------------------------
def gradients(normals, nz_min=NZ_MIN):
    """Surface slopes p = dH/dx, q = dH/dy from n ~ (-H_x, -H_y, 1), n_z clamped below."""
    n = np.asarray(normals, np.float64)
    nz = np.maximum(n[..., 2], nz_min)
    return -n[..., 0] / nz, -n[..., 1] / nz


def poisson_rhs(p, q, h):
    """b = D^T g of the edge least-squares problem, trapezoidal edge targets
    g = h (p_a + p_b) / 2 on row edges and h (q_a + q_b) / 2 on column edges."""
    H, W = p.shape
    gh = h * (p[:, :-1] + p[:, 1:]) / 2.0
    gv = h * (q[:-1, :] + q[1:, :]) / 2.0
    b = np.zeros((H, W))
    b[:, 1:] += gh
    b[:, :-1] -= gh
    b[1:, :] += gv
    b[:-1, :] -= gv
    return b


def laplacian_apply(x):
    """Neumann 5-point graph Laplacian (degree minus neighbours) of an (H, W) array."""
    y = np.zeros_like(x, dtype=np.float64)
    dx = x[:, 1:] - x[:, :-1]
    dy = x[1:, :] - x[:-1, :]
    y[:, :-1] -= dx
    y[:, 1:] += dx
    y[:-1, :] -= dy
    y[1:, :] += dy
    return y


def poisson_solve(normals, h, nz_min=NZ_MIN):
    """Depth minimising sum over edges (H_b - H_a - g_e)^2 with mean(H) = 0.

    The normal equations L H = b use the Neumann graph Laplacian of the pixel grid;
    its eigenvectors are the products of DCT-II cosines with eigenvalues
    (2 - 2cos(pi k / H)) + (2 - 2cos(pi l / W)), so the exact solution is a scaled
    pair of orthonormal cosine transforms; the constant mode is set to zero."""
    p, q = gradients(normals, nz_min)
    H, W = p.shape
    b = poisson_rhs(p, q, h)
    B = dctn(b, type=2, norm="ortho")
    lam = (2.0 - 2.0 * np.cos(np.pi * np.arange(H) / H))[:, None] + \
          (2.0 - 2.0 * np.cos(np.pi * np.arange(W) / W))[None, :]
    lam[0, 0] = 1.0
    X = B / lam
    X[0, 0] = 0.0
    return idctn(X, type=2, norm="ortho")


def edge_slope_residuals(depth, normals, h, nz_min=NZ_MIN):
    """Slope residual of every grid edge: u = (H_b - H_a) / h - (s_a + s_b) / 2 with s the
    slope p along rows (edges (i, j)-(i, j+1), shape (H, W-1)) and q along columns (shape (H-1, W))."""
    d = np.asarray(depth, np.float64)
    p, q = gradients(normals, nz_min)
    uh = (d[:, 1:] - d[:, :-1]) / h - (p[:, :-1] + p[:, 1:]) / 2.0
    uv = (d[1:, :] - d[:-1, :]) / h - (q[:-1, :] + q[1:, :]) / 2.0
    return uh, uv


def huber_weights(u, delta):
    """IRLS weight of the Huber M-estimator: 1 where |u| <= delta, delta / |u| beyond."""
    a = np.abs(np.asarray(u, np.float64))
    return np.where(a <= delta, 1.0, delta / np.maximum(a, 1e-300))


def weighted_poisson_solve(normals, h, wh, wv, nz_min=NZ_MIN):
    """Depth minimising sum wh (H_{i,j+1} - H_ij - gh)^2 + sum wv (H_{i+1,j} - H_ij - gv)^2,
    mean(H) = 0, with the trapezoidal targets of poisson_rhs; wh (H, W-1), wv (H-1, W) > 0.
    Sparse normal equations, solved directly with node 0 held at 0, then centred."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.linalg import spsolve
    p, q = gradients(normals, nz_min)
    H, W = p.shape
    idx = np.arange(H * W).reshape(H, W)
    wh = np.asarray(wh, np.float64)
    wv = np.asarray(wv, np.float64)
    gh = h * (p[:, :-1] + p[:, 1:]) / 2.0
    gv = h * (q[:-1, :] + q[1:, :]) / 2.0
    a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])  # edge tails
    b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])    # edge heads
    w = np.concatenate([wh.ravel(), wv.ravel()])
    g = np.concatenate([gh.ravel(), gv.ravel()])
    rows = np.concatenate([a, b, a, b])
    cols = np.concatenate([a, b, b, a])
    vals = np.concatenate([w, w, -w, -w])
    L = coo_matrix((vals, (rows, cols)), shape=(H * W, H * W)).tocsr()
    rhs = np.zeros(H * W)
    np.add.at(rhs, b, w * g)
    np.add.at(rhs, a, -w * g)
    x = np.zeros(H * W)
    x[1:] = spsolve(L[1:, 1:].tocsc(), rhs[1:])
    x -= x.mean()
    return x.reshape(H, W)


def irls_solve(normals, h, delta, iters, nz_min=NZ_MIN):
    """Integration by the Huber M-estimator (the robust estimator the paper names for this
    step), by iteratively reweighted least squares: H^0 is the least-squares surface;
    H^i solves the weighted problem with the Huber weights of the slope residuals of
    H^(i-1) (threshold `delta` in slope units)."""
    d = poisson_solve(normals, h, nz_min)
    for _ in range(iters):
        uh, uv = edge_slope_residuals(d, normals, h, nz_min)
        d = weighted_poisson_solve(normals, h, huber_weights(uh, delta), huber_weights(uv, delta), nz_min)
    return d


def diff_norm(h_new, h_old):
    """D_H: max |H_{t+1} - H_t| over the depth range of H_{t+1}, and the RMS difference."""
    a = np.asarray(h_new, np.float64)
    b = np.asarray(h_old, np.float64)
    d = a - b
    rng = a.max() - a.min()
    return (np.abs(d).max() / rng if rng > 0 else 0.0), float(np.sqrt((d * d).mean()))


# ----------------------------------------------------------------------------
# The loop
# ----------------------------------------------------------------------------
def ps_step(A0, rho_t, lbar, lights, tau_lo=TAU_LO, tau_hi=TAU_HI, cond_max=COND_MAX):
    """Subtract + PS for (K, C, H, W) images; rho_t (C, P), lbar (K, C, P)."""
    K, C, H, W = A0.shape
    A = np.asarray(A0).reshape(K, C, -1)
    v = valid_rows(A, rho_t, lbar, tau_lo, tau_hi)
    I = correct_images(A, rho_t, lbar)
    return ps_solve(I, v, lights, cond_max)


def irtps_run(A0, lights, env, n_iter, spp, bounces, seed, *, shadow_rays=True, fp32=True, threads=0,
              tau_lo=TAU_LO, tau_hi=TAU_HI, obj=0, shared=False, irls_iters=0, irls_delta=0.05,
              fill_holes=False):
    """The IRT-PS loop: iteration 0 is classic PS + integration; each further
    iteration traces Lbar on the current estimate (iteration index t), subtracts
    rho_t * Lbar_t from the ORIGINAL images, re-solves PS and re-integrates.
    `obj` is the object index in the Philox key {seed_lo ^ obj, seed_hi}; `shared`
    selects light-shared sampling for the trace; irls_iters > 0 integrates with the
    Huber M-estimator (irls_solve) instead of plain least squares; fill_holes
    replaces Lbar at the holes of each light's trace (hole_mask) by the non-uniform
    interpolation of its known pixels (interpolate_holes; the single-sample variant,
    per-light sampling).
    Returns a list of per-iteration dicts (depth, normals, albedo, lbar, dH)."""
    A0 = np.asarray(A0, np.float32)
    K, C, H, W = A0.shape
    h = 1.0 / W
    zero = np.zeros((K, C, H * W))
    def integrate(nn):
        if irls_iters > 0:
            return irls_solve(nn.reshape(H, W, 3), h, irls_delta, irls_iters)
        return poisson_solve(nn.reshape(H, W, 3), h)

    n, rho, ok = ps_step(A0, np.zeros((C, H * W)), zero, lights, tau_lo, tau_hi)
    depth = integrate(n)
    hist = [dict(depth=depth, normals=n.reshape(H, W, 3), albedo=rho.reshape(C, H, W), ok=ok,
                 lbar=None, dH=None, counts=(0, 0))]
    for t in range(n_iter):
        st = hist[-1]
        lbar, rec, counts = trace(st["depth"].astype(np.float32), st["normals"].astype(np.float32),
                                  st["albedo"].astype(np.float32), lights, env, spp, bounces, seed, t,
                                  obj=obj, shadow_rays=shadow_rays, fp32=fp32, threads=threads, shared=shared,
                                  records=fill_holes)
        if fill_holes:
            if shared:
                raise ValueError("hole filling follows per-light sampling")
            known = ~hole_mask(rec).reshape(K, H, W)
            lbar = interpolate_holes(lbar.reshape(K, C, H, W), known).reshape(K, C, H * W)
        n, rho, ok = ps_step(A0, st["albedo"].astype(np.float32).reshape(C, -1), lbar, lights, tau_lo,
                             tau_hi)
        depth = integrate(n)
        hist.append(dict(depth=depth, normals=n.reshape(H, W, 3), albedo=rho.reshape(C, H, W), ok=ok,
                         lbar=lbar.reshape(K, C, H, W), dH=diff_norm(depth, st["depth"]), counts=counts))
    return hist


# ----------------------------------------------------------------------------
# Evaluation (Sec. V) and parity measures
# ----------------------------------------------------------------------------
def height_error(h_gt, h):
    """Mean |H_GT - H_t| after removing each surface's mean (heights are defined up to a constant)."""
    a = np.asarray(h_gt, np.float64)
    b = np.asarray(h, np.float64)
    return float(np.abs((a - a.mean()) - (b - b.mean())).mean())


def albedo_error(rho_gt, rho):
    """Mean over channels of the per-channel mean absolute albedo error."""
    a = np.asarray(rho_gt, np.float64)
    b = np.asarray(rho, np.float64)
    return float(np.mean([np.abs(a[c] - b[c]).mean() for c in range(a.shape[0])]))


def normal_error(n_gt, n):
    """Mean over x, y, z of the per-axis mean absolute normal error."""
    a = np.asarray(n_gt, np.float64).reshape(-1, 3)
    b = np.asarray(n, np.float64).reshape(-1, 3)
    return float(np.mean([np.abs(a[:, i] - b[:, i]).mean() for i in range(3)]))


def angular_error_deg(a, b):
    """Per-pixel angle between normals, atan2(|a x b|, a . b), in degrees."""
    a = np.asarray(a, np.float64).reshape(-1, 3)
    b = np.asarray(b, np.float64).reshape(-1, 3)
    cr = np.cross(a, b)
    return np.degrees(np.arctan2(np.sqrt((cr * cr).sum(axis=1)), (a * b).sum(axis=1)))
