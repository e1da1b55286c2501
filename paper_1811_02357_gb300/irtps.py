"""Thin Python binding of the IRT-PS C ABI (include/irtps.h).

Argument marshalling only: every step of the method runs in the CUDA library
`_lib/libirtps.so`.  Host arrays are numpy arrays; device arrays are anything
exposing `data_ptr()` (torch tensors) or a raw integer address.  There is no
CPU fallback: if the library is missing or fails to load, importing this
module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libirtps.so")

IRTPS_OK = 0
IRTPS_EINVAL = -1
IRTPS_ENOMEM = -2
IRTPS_ECUDA = -3
IRTPS_ENOTREADY = -4
IRTPS_ETIMEOUT = -5
IRTPS_ENUMERIC = -6
IRTPS_F32 = 0
IRTPS_F16 = 1
NOALLOC_MAX_PIXELS = 512 * 512  # grid size limit of irtps_integrate_noalloc
FORWARD_ITER = 0xFFFFFFFF

EXPORTED = [
    "irtps_default_options", "irtps_create", "irtps_set_stream", "irtps_set_images", "irtps_iterate",
    "irtps_trace", "irtps_solve_normals", "irtps_integrate", "irtps_trace_pixels", "irtps_set_state",
    "irtps_set_indirect", "irtps_render", "irtps_get_normals", "irtps_get_albedo", "irtps_get_depth",
    "irtps_get_indirect", "irtps_get_valid", "irtps_get_holes", "irtps_get_stats", "irtps_probe_dirs",
    "irtps_probe_rays", "irtps_interpolate_holes",
    "irtps_last_error", "irtps_destroy", "irtps_integrate_noalloc", "irtps_set_object", "irtps_set_tuning",
    "irtps_get_tuning", "irtps_autotune", "irtps_set_ps_tuning", "irtps_get_ps_tuning", "irtps_batch_create", "irtps_batch_set_stream", "irtps_batch_set_images", "irtps_batch_iterate", "irtps_batch_get_stats",
    "irtps_batch_set_tuning", "irtps_batch_get_tuning", "irtps_batch_autotune", "irtps_batch_last_error",
    "irtps_batch_destroy",
]


class irtps_options(ctypes.Structure):
    _fields_ = [("shadow_rays", ctypes.c_int), ("tau_lo", ctypes.c_float), ("tau_hi", ctypes.c_float),
                ("cond_max", ctypes.c_double), ("nz_min", ctypes.c_float), ("cg_tol", ctypes.c_double),
                ("cg_max_iter", ctypes.c_int), ("cg_check_every", ctypes.c_int), ("stop_tol", ctypes.c_double),
                ("precond", ctypes.c_int), ("use_graph", ctypes.c_int), ("sampling", ctypes.c_int),
                ("irls_iters", ctypes.c_int), ("irls_delta", ctypes.c_float), ("early_escape", ctypes.c_int),
                ("fill_holes", ctypes.c_int), ("ps_tensor", ctypes.c_int)]


class irtps_stats(ctypes.Structure):
    _fields_ = [("primary_segments", ctypes.c_ulonglong), ("segments", ctypes.c_ulonglong),
                ("walk_overflows", ctypes.c_ulonglong), ("cg_iterations", ctypes.c_int),
                ("cg_rel_residual", ctypes.c_double), ("dH_max", ctypes.c_double), ("dH_rms", ctypes.c_double),
                ("iterations_done", ctypes.c_int), ("node_visits", ctypes.c_ulonglong),
                ("tri_tests", ctypes.c_ulonglong), ("trace_ms", ctypes.c_double), ("ps_ms", ctypes.c_double),
                ("depth_ms", ctypes.c_double), ("launches", ctypes.c_ulonglong), ("draws", ctypes.c_ulonglong),
                ("fill_ms", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class IrtpsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"irtps error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                          f"g.build()'` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, u32, u64, f32, dbl = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_float, ctypes.c_double)
    sig = {
        "irtps_default_options": (None, [P]),
        "irtps_create": (i32, [P, i32, i32, i32, i32, P, P, i32, i32, P]),
        "irtps_set_stream": (i32, [P, P]),
        "irtps_set_images": (i32, [P, P, i32, i32]),
        "irtps_iterate": (i32, [P, i32, i32, i32, u64, P]),
        "irtps_trace": (i32, [P, i32, i32, u64, u32, u32]),
        "irtps_solve_normals": (i32, [P]),
        "irtps_integrate": (i32, [P]),
        "irtps_trace_pixels": (i32, [P, P, i32, i32, i32, u64, u32, u32, P, P]),
        "irtps_set_state": (i32, [P, P, P, P]),
        "irtps_set_indirect": (i32, [P, P]),
        "irtps_render": (i32, [P, i32, i32, u64, f32, P, i32]),
        "irtps_get_normals": (i32, [P, P, i32]),
        "irtps_get_albedo": (i32, [P, P, i32]),
        "irtps_get_depth": (i32, [P, P, i32]),
        "irtps_get_indirect": (i32, [P, P, i32]),
        "irtps_get_valid": (i32, [P, P, i32]),
        "irtps_get_holes": (i32, [P, P, i32]),
        "irtps_interpolate_holes": (i32, [P, P, i32, i32, i32, i32]),
        "irtps_get_stats": (i32, [P, P]),
        "irtps_probe_dirs": (i32, [i32, P, P, P, P]),
        "irtps_probe_rays": (i32, [P, i32, P, P, P]),
        "irtps_last_error": (ctypes.c_char_p, [P]),
        "irtps_integrate_noalloc": (i32, [P, i32, i32, f32, dbl, i32, P, P]),
        "irtps_destroy": (None, [P]),
        "irtps_set_object": (i32, [P, u32]),
        "irtps_set_tuning": (i32, [P, i32, i32]),
        "irtps_get_tuning": (i32, [P, P, P]),
        "irtps_set_ps_tuning": (i32, [P, i32]),
        "irtps_get_ps_tuning": (i32, [P, P]),
        "irtps_autotune": (i32, [P, i32, i32, u64, P]),
        "irtps_batch_create": (i32, [P, P, i32, i32]),
        "irtps_batch_iterate": (i32, [P, i32, P, P, u64, P]),
        "irtps_batch_set_stream": (i32, [P, P]),
        "irtps_batch_set_images": (i32, [P, P, i32, i32]),
        "irtps_batch_get_stats": (i32, [P, P]),
        "irtps_batch_set_tuning": (i32, [P, i32, i32]),
        "irtps_batch_get_tuning": (i32, [P, P, P]),
        "irtps_batch_autotune": (i32, [P, P, P, u64, P]),
        "irtps_batch_last_error": (ctypes.c_char_p, [P]),
        "irtps_batch_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _addr(a):
    """Address of a numpy array (host), a torch tensor (data_ptr) or an int."""
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(handle, rc):
    if rc != IRTPS_OK:
        msg = _lib.irtps_last_error(handle).decode() if handle else ""
        raise IrtpsError(rc, msg)


# ---------------------------------------------------------------------------
# C-ABI names, one to one
# ---------------------------------------------------------------------------
def irtps_default_options():
    opt = irtps_options()
    _lib.irtps_default_options(ctypes.byref(opt))
    return opt


def irtps_create(H, W, K, C, lights, env, opt=None):
    """Returns an opaque handle (ctypes.c_void_p)."""
    l = _host(lights, np.float32).reshape(-1, 3)
    e = _host(env, np.float32)
    EH, EW = e.shape[-2], e.shape[-1]
    h = ctypes.c_void_p()
    rc = _lib.irtps_create(ctypes.byref(h), H, W, K, C, _addr(l), _addr(e), EH, EW,
                           ctypes.byref(opt) if opt is not None else None)
    if rc != IRTPS_OK:
        msg = _lib.irtps_last_error(h).decode() if h.value else ""
        if h.value:
            _lib.irtps_destroy(h)
        raise IrtpsError(rc, msg)
    return h


def irtps_set_stream(h, stream):
    _check(h, _lib.irtps_set_stream(h, ctypes.c_void_p(stream)))


def irtps_set_images(h, images, dtype=IRTPS_F32, on_device=False):
    if not on_device:
        images = _host(images, np.float16 if dtype == IRTPS_F16 else np.float32)
    _check(h, _lib.irtps_set_images(h, _addr(images), dtype, int(on_device)))


def irtps_iterate(h, n_iter, spp, bounces, seed):
    dh = ctypes.c_double(0.0)
    _check(h, _lib.irtps_iterate(h, n_iter, spp, bounces, seed, ctypes.byref(dh)))
    return dh.value


def irtps_trace(h, spp, bounces, seed, iteration, stream_tag=0):
    _check(h, _lib.irtps_trace(h, spp, bounces, seed, iteration & 0xFFFFFFFF, stream_tag))


def irtps_solve_normals(h):
    _check(h, _lib.irtps_solve_normals(h))


def irtps_integrate(h):
    _check(h, _lib.irtps_integrate(h))


def irtps_trace_pixels(h, pixels, K, C, spp, bounces, seed, iteration, stream_tag=0, records=False,
                       shared=False):
    """`shared`: the context uses light-shared sampling (records (n_pix, spp, bounces, 1 + K))."""
    pix = _host(pixels, np.int32)
    out = np.zeros((K, C, pix.size), np.float32)
    shape = (pix.size, spp, bounces, 1 + K) if shared else (pix.size, K, spp, bounces, 2)
    rec = np.zeros(shape, np.int32) if records else None
    _check(h, _lib.irtps_trace_pixels(h, _addr(pix), pix.size, spp, bounces, seed, iteration & 0xFFFFFFFF,
                                      stream_tag, _addr(out), _addr(rec)))
    return out, rec


def irtps_set_state(h, depth=None, normals=None, albedo=None):
    d = None if depth is None else _host(depth, np.float32)
    n = None if normals is None else _host(normals, np.float32)
    a = None if albedo is None else _host(albedo, np.float32)
    _check(h, _lib.irtps_set_state(h, _addr(d), _addr(n), _addr(a)))


def irtps_set_indirect(h, indirect):
    _check(h, _lib.irtps_set_indirect(h, _addr(_host(indirect, np.float32))))


def irtps_render(h, shape, spp, bounces, seed, sigma, out=None):
    """Host render unless `out` (a device tensor) is given."""
    if out is None:
        buf = np.zeros(shape, np.float32)
        _check(h, _lib.irtps_render(h, spp, bounces, seed, sigma, _addr(buf), 0))
        return buf
    _check(h, _lib.irtps_render(h, spp, bounces, seed, sigma, _addr(out), 1))
    return out


def _get(fn, h, shape, dtype, out):
    if out is None:
        buf = np.zeros(shape, dtype)
        _check(h, fn(h, _addr(buf), 0))
        return buf
    _check(h, fn(h, _addr(out), 1))
    return out


def irtps_get_normals(h, shape, out=None):
    return _get(_lib.irtps_get_normals, h, shape, np.float32, out)


def irtps_get_albedo(h, shape, out=None):
    return _get(_lib.irtps_get_albedo, h, shape, np.float32, out)


def irtps_get_depth(h, shape, out=None):
    return _get(_lib.irtps_get_depth, h, shape, np.float32, out)


def irtps_get_indirect(h, shape, out=None):
    return _get(_lib.irtps_get_indirect, h, shape, np.float32, out)


def irtps_get_valid(h, shape, out=None):
    return _get(_lib.irtps_get_valid, h, shape, np.uint8, out)


def irtps_get_holes(h, shape, out=None):
    return _get(_lib.irtps_get_holes, h, shape, np.uint8, out)


def irtps_interpolate_holes(values, holes):
    """Non-uniform interpolation of the holes of a (K, C, H, W) float32 stack; holes (K, H, W),
    nonzero = missing.  Returns the filled copy."""
    v = np.array(_host(values, np.float32), np.float32, order="C", copy=True)
    K, C, H, W = v.shape
    m = _host(holes, np.uint8).reshape(K, H, W)
    rc = _lib.irtps_interpolate_holes(_addr(v), _addr(m), K, C, H, W)
    if rc != IRTPS_OK:
        raise IrtpsError(rc, "interpolate_holes")
    return v


def irtps_get_stats(h):
    s = irtps_stats()
    _check(h, _lib.irtps_get_stats(h, ctypes.byref(s)))
    return s.as_dict()


def irtps_probe_dirs(normals, x0, x1):
    n = _host(normals, np.float32).reshape(-1, 3)
    a = _host(x0, np.uint32)
    b = _host(x1, np.uint32)
    out = np.zeros_like(n)
    rc = _lib.irtps_probe_dirs(n.shape[0], _addr(n), _addr(a), _addr(b), _addr(out))
    if rc != IRTPS_OK:
        raise IrtpsError(rc, "probe_dirs")
    return out


def irtps_probe_rays(h, rays):
    r = _host(rays, np.float32).reshape(-1, 6)
    t = np.zeros(r.shape[0], np.float32)
    tri = np.zeros(r.shape[0], np.int32)
    _check(h, _lib.irtps_probe_rays(h, r.shape[0], _addr(r), _addr(t), _addr(tri)))
    return t, tri


def _device_f32(t, n, name, align=4):
    """A CUDA float32 tensor, contiguous, with at least n elements and `align`-byte aligned (the
    kernels read past no end of it); raises before the C call otherwise."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name}: need a contiguous float32 CUDA tensor")
    if t.numel() < n:
        raise ValueError(f"{name}: {t.numel()} elements, need {n}")
    if t.data_ptr() % align:
        raise ValueError(f"{name}: address not {align}-byte aligned")


def irtps_integrate_noalloc(normals, depth, H, W, nz_min=0.05, tol=1e-9, max_iter=50000, stream=0):
    """Allocation-free depth solve on device buffers: normals (H, W, 4) float32, depth (H, W) float32
    (warm start in, surface out).  `stream` is a raw cudaStream_t value (0: legacy default stream)."""
    runs = H >= 2 and W >= 2 and H * W <= NOALLOC_MAX_PIXELS  # else the library rejects the sizes itself
    _device_f32(normals, 4 * H * W if runs else 0, "normals", 16)  # read as float4
    _device_f32(depth, H * W if runs else 0, "depth")
    rc = _lib.irtps_integrate_noalloc(_addr(normals), H, W, nz_min, tol, max_iter, _addr(depth),
                                      ctypes.c_void_p(stream))
    if rc != IRTPS_OK:
        raise IrtpsError(rc, "integrate_noalloc")


def irtps_last_error(h):
    return _lib.irtps_last_error(h).decode()


def irtps_set_object(h, obj):
    _check(h, _lib.irtps_set_object(h, obj))


def irtps_set_tuning(h, blocks_per_sm, mip_cut):
    _check(h, _lib.irtps_set_tuning(h, blocks_per_sm, mip_cut))


def irtps_set_ps_tuning(h, pixels_per_thread):
    _check(h, _lib.irtps_set_ps_tuning(h, pixels_per_thread))


def irtps_get_ps_tuning(h):
    v = ctypes.c_int(0)
    _check(h, _lib.irtps_get_ps_tuning(h, ctypes.byref(v)))
    return v.value


def irtps_get_tuning(h):
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(h, _lib.irtps_get_tuning(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def irtps_autotune(h, spp_probe, bounces, seed):
    ms = ctypes.c_double(0.0)
    _check(h, _lib.irtps_autotune(h, spp_probe, bounces, seed, ctypes.byref(ms)))
    return ms.value


def _check_batch(b, rc):
    if rc != IRTPS_OK:
        msg = _lib.irtps_batch_last_error(b).decode() if b else ""
        raise IrtpsError(rc, msg)


def irtps_batch_create(handles, use_graph=False):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    b = ctypes.c_void_p()
    rc = _lib.irtps_batch_create(ctypes.byref(b), arr, len(handles), 1 if use_graph else 0)
    if rc != IRTPS_OK:
        raise IrtpsError(rc, "batch_create")
    return b


def irtps_batch_set_stream(b, stream):
    _check_batch(b, _lib.irtps_batch_set_stream(b, ctypes.c_void_p(stream) if stream else None))


def irtps_batch_set_images(b, images, dtype=IRTPS_F32, on_device=False):
    """images: one array per object (numpy host arrays, or device tensors with on_device)."""
    if not on_device:
        images = [_host(a, np.float16 if dtype == IRTPS_F16 else np.float32) for a in images]
    ptrs = (ctypes.c_void_p * len(images))(*[_addr(a).value for a in images])
    _check_batch(b, _lib.irtps_batch_set_images(b, ptrs, dtype, 1 if on_device else 0))


def irtps_batch_iterate(b, n_iter, spp, bounces, seed):
    n = len(spp)
    s = _host(spp, np.int32)
    r = _host(bounces, np.int32)
    dh = np.zeros(n, np.float64)
    _check_batch(b, _lib.irtps_batch_iterate(b, n_iter, _addr(s), _addr(r), seed, _addr(dh)))
    return dh


def irtps_batch_get_stats(b):
    st = irtps_stats()
    _check_batch(b, _lib.irtps_batch_get_stats(b, ctypes.byref(st)))
    return st.as_dict()


def irtps_batch_set_tuning(b, blocks_per_sm, mip_cut):
    _check_batch(b, _lib.irtps_batch_set_tuning(b, blocks_per_sm, mip_cut))


def irtps_batch_get_tuning(b):
    x, y = ctypes.c_int(0), ctypes.c_int(0)
    _check_batch(b, _lib.irtps_batch_get_tuning(b, ctypes.byref(x), ctypes.byref(y)))
    return x.value, y.value


def irtps_batch_autotune(b, spp_probe, bounces, seed):
    s = _host(spp_probe, np.int32)
    r = _host(bounces, np.int32)
    ms = ctypes.c_double(0.0)
    _check_batch(b, _lib.irtps_batch_autotune(b, _addr(s), _addr(r), seed, ctypes.byref(ms)))
    return ms.value


def irtps_batch_last_error(b):
    return _lib.irtps_batch_last_error(b).decode()


def irtps_batch_destroy(b):
    if b is not None and b.value:
        _lib.irtps_batch_destroy(b)


def irtps_destroy(h):
    if h is not None and h.value:
        _lib.irtps_destroy(h)


# ---------------------------------------------------------------------------
# Convenience wrapper (same calls, shapes remembered)
# ---------------------------------------------------------------------------
class Context:
    """One IRT-PS object: H x W pixels, K lights, C channels (1 or 3)."""

    def __init__(self, H, W, lights, env, opt=None):
        lights = np.asarray(lights, np.float32).reshape(-1, 3)
        env = np.asarray(env, np.float32)
        self.H, self.W, self.K, self.C = H, W, lights.shape[0], env.shape[0]
        self.shared = bool(opt is not None and opt.sampling == 1)
        self.h = irtps_create(H, W, self.K, self.C, lights, env, opt)

    def close(self):
        irtps_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        irtps_set_stream(self.h, stream)

    def set_images(self, images, dtype=IRTPS_F32, on_device=False):
        irtps_set_images(self.h, images, dtype, on_device)

    def iterate(self, n_iter, spp, bounces, seed):
        return irtps_iterate(self.h, n_iter, spp, bounces, seed)

    def trace(self, spp, bounces, seed, iteration, stream_tag=0):
        irtps_trace(self.h, spp, bounces, seed, iteration, stream_tag)

    def solve_normals(self):
        irtps_solve_normals(self.h)

    def integrate(self):
        irtps_integrate(self.h)

    def trace_pixels(self, pixels, spp, bounces, seed, iteration, stream_tag=0, records=False):
        return irtps_trace_pixels(self.h, pixels, self.K, self.C, spp, bounces, seed, iteration, stream_tag,
                                  records, self.shared)

    def set_state(self, depth=None, normals=None, albedo=None):
        irtps_set_state(self.h, depth, normals, albedo)

    def set_indirect(self, indirect):
        irtps_set_indirect(self.h, indirect)

    def render(self, spp, bounces, seed, sigma, out=None):
        return irtps_render(self.h, (self.K, self.C, self.H, self.W), spp, bounces, seed, sigma, out)

    def normals(self, out=None):
        return irtps_get_normals(self.h, (self.H, self.W, 4), out)

    def albedo(self, out=None):
        return irtps_get_albedo(self.h, (self.C, self.H, self.W), out)

    def depth(self, out=None):
        return irtps_get_depth(self.h, (self.H, self.W), out)

    def indirect(self, out=None):
        return irtps_get_indirect(self.h, (self.K, self.C, self.H, self.W), out)

    def valid(self, out=None):
        return irtps_get_valid(self.h, (self.H, self.W), out)

    def holes(self, out=None):
        return irtps_get_holes(self.h, (self.K, self.H, self.W), out)

    def stats(self):
        return irtps_get_stats(self.h)

    def probe_rays(self, rays):
        return irtps_probe_rays(self.h, rays)

    def set_object(self, obj):
        irtps_set_object(self.h, obj)

    def set_tuning(self, blocks_per_sm, mip_cut):
        irtps_set_tuning(self.h, blocks_per_sm, mip_cut)

    def tuning(self):
        return irtps_get_tuning(self.h)

    def set_ps_tuning(self, pixels_per_thread):
        irtps_set_ps_tuning(self.h, pixels_per_thread)

    def ps_tuning(self):
        return irtps_get_ps_tuning(self.h)

    def autotune(self, spp_probe, bounces, seed):
        return irtps_autotune(self.h, spp_probe, bounces, seed)


class Batch:
    """Many contexts iterated together, one launch per IRT stage.  The contexts stay owned by the
    caller and must outlive the batch; context i gets object index i."""

    def __init__(self, contexts, use_graph=False):
        self.contexts = list(contexts)
        self.b = irtps_batch_create([c.h for c in self.contexts], use_graph)

    def close(self):
        irtps_batch_destroy(self.b)
        self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "b", None) is not None:
                self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        irtps_batch_set_stream(self.b, stream)

    def set_images(self, images, dtype=IRTPS_F32, on_device=False):
        irtps_batch_set_images(self.b, images, dtype, on_device)

    def iterate(self, n_iter, spp, bounces, seed):
        return irtps_batch_iterate(self.b, n_iter, spp, bounces, seed)

    def stats(self):
        return irtps_batch_get_stats(self.b)

    def set_tuning(self, blocks_per_sm, mip_cut):
        irtps_batch_set_tuning(self.b, blocks_per_sm, mip_cut)

    def tuning(self):
        return irtps_batch_get_tuning(self.b)

    def autotune(self, spp_probe, bounces, seed):
        return irtps_batch_autotune(self.b, spp_probe, bounces, seed)
