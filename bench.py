"""IRT-PS benchmark: Mrays/s of the IRT-PS loop on one seeded synthetic workload.

Workload `bumps_2048` (default; the 2048x2048 precision configuration at its full
spec): 2048x2048 RGB heightfield of 200 Gaussian bumps and 4 concave bowls,
Voronoi albedo, 64x128 RGB cosine environment, K = 32 lights on a jittered ring,
images stored in FP16; trace 512 spp per (pixel, light), 2 bounces.  Input images
are rendered once on the GPU from the ground truth (64 spp, 2 bounces, sigma 0.002).

One step is what a user of the C ABI runs per IRT iteration: upload the images
from pinned host memory (irtps_set_images, which also runs iteration 0: classic
PS + integration), one IRT iteration (irtps_iterate: pyramid, horizon bounds,
trace, subtract + PS, integration, D_H), and read the depth, normals and albedo
back to pinned host memory.

value      = traced segments (primary, bounce and shadow rays) / second of the IRT
             iterations (CUDA events around irtps_iterate; inputs resident in HBM)
e2e        = the same segments / second of the whole step (events around all three
             calls: host->device images, iteration 0, the iteration, results back)
accuracy   = stage-wise errors against the FP64 oracle (outside the timed region):
             given the GPU's iteration-t state, the oracle traces sampled pixels,
             solves their normals from the same FP16 images, and integrates the
             GPU's normals over the whole grid
roofline   = the trace kernel (dominant): algorithmic lane operations per second
             against the lane-issue peak (bound "alu")
cpu_baseline = the oracle (plain C++) on the host cores over a pixel sample
evaluation (--evaluate) = errors against the ground truth (height, albedo, normal; the paper's
             evaluation measures) of classic PS and of IRT-PS with 1, 2 and 3 traced reflections

Other workloads: `bumps_512` (512x512 RGB bumps and a V-groove, K = 12, 256 spp,
2 bounces; one step = a 5-iteration job), `bowl_64` (64x64 bowl), `bumps_4096_spp16`
(4096x4096, K = 64 at 16 spp), `bumps_512_single` (one sample per (pixel, light),
holes filled).

Workload `batch_64`: 64 objects of scenes.batch_objects (sides log-uniform in
96..1024, K in {4, 8, 16, 32}, spp in {64, 128, 256}, bounces in {1, 2}); one
step = iteration 0 (batched set_images) and one IRT iteration of every object
through one batch (one launch per stage; timed enqueued, for its stage events, and once more with
the iteration replayed as a CUDA graph); the same job as 64 per-object contexts
iterated one after another is timed beside it.

`--impl reference` times the oracle itself on the same workload (pixel samples).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (scene factory, its arguments, spp, bounces, IRT iterations per step, render spp, render bounces)
    # the 2048x2048, K = 32 precision configuration at its full spec (FP16 images, 512 spp, 2 bounces)
    "bumps_2048": ("bumps_2048", {}, 512, 2, 1, 64, 2),
    "bumps_512": ("bumps_512", {}, 256, 2, 5, 256, 2),
    "bowl_64": ("bowl_64", {}, 64, 1, 3, 256, 1),
    # a small case of the same kernels for profiler captures (one IRT iteration per job)
    "bumps_256_profile": ("bumps_512", {"H": 256, "W": 256}, 32, 2, 1, 32, 2),
    # a small case of the 2048x2048, K = 32 kernels for profiler captures (2 spp: one trace launch
    # of about a tenth of a second)
    "bumps_2048_profile": ("bumps_2048", {}, 2, 2, 1, 4, 1),
    # the 2048x2048, K = 32 configuration at an eighth of its samples (64 spp)
    "bumps_2048_spp64": ("bumps_2048", {}, 64, 2, 1, 4, 1),
    # the 4096x4096, K = 64 configuration at a sixty-fourth of its samples (16 spp)
    "bumps_4096_spp16": ("bumps_4096", {}, 16, 2, 1, 4, 1),
    # the batched pattern: 64 objects (sides 96..1024, K, spp, bounces per object), one IRT
    # iteration of all of them per step, against per-object launches (run_batch)
    "batch_64": ("batch_objects", {}, None, None, 1, 32, 1),
    # a small batch of the same kernels for profiler captures (16 objects, sides 96..384)
    "batch_16_profile": ("batch_objects", {"n": 16, "side_hi": 384}, None, None, 1, 8, 1),
    # the single-sample variant: one path per (pixel, light), holes filled by interpolation
    "bumps_512_single": ("bumps_512", {}, 1, 2, 5, 256, 2),
}
# context options a workload sets beyond the defaults
WORKLOAD_OPTIONS = {"bumps_512_single": {"fill_holes": 1}}
# image storage of a workload when --images is not given (the precision configurations keep FP16)
WORKLOAD_IMAGES = {"bumps_2048": "f16", "bumps_2048_spp64": "f16", "bumps_2048_profile": "f16", "bumps_4096_spp16": "f16"}
# tuner probes take spp / this many samples (a few seconds of probes on the large grids)
WORKLOAD_TUNE_DIV = {"bumps_2048": 64, "bumps_2048_spp64": 8, "bumps_2048_profile": 2, "bumps_4096_spp16": 4}

# Algorithmic lane operations per unit of trace work (counted from the formulas:
# Philox4x32-10 = 10 rounds x (2 mul.hi + 2 mul.lo + 4 xor) + 9 x 2 key adds;
# cosine direction = uniforms, 2 sqrt, turn sine/cosine polynomial, Duff basis,
# basis combination; node visit = node bounds, two exit parameters, height at the
# entry, compare; triangle test = Moeller-Trumbore with its four rejections).
OPS_PER_DRAW = 98 + 47
OPS_PER_NODE = 16
OPS_PER_TRI = 57
LANES_PER_SM = 128
# DRAM bytes (read + write) of one trace launch, per workload and sampling, from ncu captures of the
# same kernel; None where no capture of the current kernel exists
TRACE_DRAM_BYTES = {}


def sm_max_mhz():
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.split()
        return float(out[0])
    except Exception:
        return 2070.0


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=10)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def gt_errors(sc, depth, normals, albedo):
    """Errors of an estimate against the synthetic ground truth, as the paper's evaluation reports
    them: mean |H_gt - H| with each surface's mean removed, mean absolute albedo error (over channels),
    mean absolute normal-component error (over x, y, z); plus the mean angle between normals (deg)."""
    a = sc.depth.astype(np.float64)
    b = depth.astype(np.float64)
    e_h = float(np.abs((a - a.mean()) - (b - b.mean())).mean())
    e_rho = float(np.abs(sc.albedo.astype(np.float64) - albedo.astype(np.float64)).mean(axis=(1, 2)).mean())
    ng = sc.normals.reshape(-1, 3).astype(np.float64)
    ne = normals[..., :3].reshape(-1, 3).astype(np.float64)
    e_n = float(np.abs(ng - ne).mean(axis=0).mean())
    cross = np.linalg.norm(np.cross(ng, ne), axis=1)
    ang = float(np.degrees(np.arctan2(cross, (ng * ne).sum(axis=1))).mean())
    return {"height": e_h, "albedo": e_rho, "normal": e_n, "normal_deg": ang}


def evaluate(irtps, sc, spp, n_iter, seed, opt, stream, dev, render_spp=None):
    """Classic PS and IRT-PS with r = 1, 2, 3 traced reflections on images rendered with three
    (render_spp samples per pixel and light for the images, default spp)."""
    import torch
    K, C, H, W = sc.K, sc.C, sc.H, sc.W
    A = torch.empty((K, C, H, W), dtype=torch.float32, device=dev)
    with irtps.Context(H, W, sc.lights, sc.env) as gt:
        gt.set_stream(stream.cuda_stream)
        gt.set_state(sc.depth, sc.normals, sc.albedo)
        rs = render_spp or spp
        gt.render(rs, 3, 2000, 0.002, out=A)
    torch.cuda.synchronize()
    out = {"images": f"rendered with 3 reflections, {rs} spp, sigma 0.002", "irt_iterations": n_iter,
           "trace_spp": spp}
    variants = [("", opt)]
    if opt.fill_holes:  # the same loop without the hole interpolation, for comparison
        plain = irtps.irtps_options.from_buffer_copy(opt)
        plain.fill_holes = 0
        variants.append(("_no_fill", plain))
    for suffix, o in variants:
        for r in (1, 2, 3):
            with irtps.Context(H, W, sc.lights, sc.env, o) as ctx:
                ctx.set_stream(stream.cuda_stream)
                ctx.set_images(A, on_device=True)
                if r == 1 and not suffix:
                    out["classic_ps"] = gt_errors(sc, ctx.depth(), ctx.normals(), ctx.albedo())
                ctx.iterate(n_iter, spp, r, seed)
                out[f"irtps_r{r}{suffix}"] = gt_errors(sc, ctx.depth(), ctx.normals(), ctx.albedo())
    return out


def combine_ranks(ms, units, world, device):
    """Whole-job figures of N replica ranks: the slowest rank's time (max) and the units all ranks
    processed (sum).  Any process group works (nccl on GPUs; gloo in the CPU tests)."""
    if world <= 1:
        return float(ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def split_objects(costs, world):
    """Cost-balanced split of a batch's objects over ranks: objects in order of decreasing cost
    (ties by index), each to the rank whose total is smallest so far (ties to the lower rank).
    Returns each rank's object indices, ascending."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_objects(local, sizes, parts, world, rank, device):
    """One collective at the end of a split batch job: every rank contributes the float32 results
    of its own objects (local: object index -> 1-D array of sizes[index] values); rank 0 returns
    {index: array} for every object, the other ranks None.  The objects of rank r are packed in
    ascending order, padded to the longest rank's length, and all ranks' buffers exchanged by one
    all_gather (any backend: nccl on GPUs, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    lengths = [sum(sizes[i] for i in p) for p in parts]
    n = max(lengths) if lengths else 0
    buf = torch.zeros(n, dtype=torch.float32, device=device)
    off = 0
    for i in parts[rank]:
        buf[off:off + sizes[i]] = torch.as_tensor(np.asarray(local[i], np.float32).ravel(), device=device)
        off += sizes[i]
    if world > 1:
        bufs = [torch.empty(n, dtype=torch.float32, device=device) for _ in range(world)]
        dist.all_gather(bufs, buf)
    else:
        bufs = [buf]
    if rank != 0:
        return None
    out = {}
    for r, p in enumerate(parts):
        b = bufs[r].cpu().numpy()
        off = 0
        for i in p:
            out[i] = b[off:off + sizes[i]].copy()
            off += sizes[i]
    return out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(sc, spp, bounces, target_s=12.0, seed=1, shared=False, single_thread=False):
    """The oracle as it stands, on all host cores, over a pixel sample of the workload
    (`shared`: its light-shared trace; `single_thread`: also its rate on one core)."""
    import oracle
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(123)
    P = sc.H * sc.W

    def run(n):
        pix = np.sort(rng.choice(P, n, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        _, _, (prim, segs) = oracle.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, spp, bounces, seed,
                                          0, pixels=pix, fp32=True, threads=threads, shared=shared)
        return time.perf_counter() - t0, segs

    n = max(threads, 16)
    dt, segs = run(n)
    while dt < 0.25 * target_s and n < P:  # grow the pilot until its rate is representative
        n = int(min(P, n * max(2.0, 0.5 * target_s / max(dt, 1e-3))))
        dt, segs = run(n)
    n2 = int(min(P, max(n, n * target_s / max(dt, 1e-3))))
    if n2 > n:
        dt, segs = run(n2)
    else:
        n2 = n
    out = {"value": segs / dt / 1e6, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
           "sample": f"{n2} random pixels of the workload x {'one path for all ' if shared else ''}{sc.K} lights "
                     f"x {spp} spp x {bounces} bounces "
                     f"(ground-truth state, one trace pass, {segs} segments, {dt:.1f} s)"}
    if single_thread and threads > 1:  # the oracle's other mode: one core, about 3 s of work
        n1 = int(max(1, min(P, n2 * 3.0 / max(dt * threads, 1e-3))))
        pix = np.sort(rng.choice(P, n1, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        _, _, (_, segs1) = oracle.trace(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, spp, bounces, seed, 0,
                                        pixels=pix, fp32=True, threads=1, shared=shared)
        dt1 = time.perf_counter() - t0
        out["single_thread"] = {"value": segs1 / dt1 / 1e6, "unit": "Mrays/s", "cores": 1,
                                "sample": f"{n1} random pixels, {segs1} segments, {dt1:.1f} s"}
    return out


# the library's default early-escape option (irtps_default_options), for the reference arm's config
DEFAULT_EARLY_ESCAPE = 2


def single_config(args, H, W, K, C, spp, bounces, n_iter, early_escape, world):
    """The workload part of a single-object line's config, the same in both arms."""
    big = K * C * H * W * (2 if args.images == "f16" else 4) > 256 * 1024 * 1024
    return {"workload": args.workload, "H": H, "W": W, "K": K, "C": C, "spp": spp, "images": args.images,
            "sampling": args.sampling,
            "options": dict(WORKLOAD_OPTIONS.get(args.workload, {}), early_escape=early_escape),
            "bounces": bounces, "irt_iterations_per_step": n_iter, "parallelism": f"replicas{world}",
            "l2": ("inputs larger than L2 (the step's images, copied in every step)" if big else
                   "512 MB buffer written between timed steps")}


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, same workload and metric."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import scenes
    name, kw, spp, bounces, n_iter, _, _ = WORKLOADS[args.workload]
    if name == "batch_objects":  # a sample of the first object (the oracle traces one object at a time)
        sc, spp, bounces = scenes.batch_objects(n=1)[0]
    else:
        sc = getattr(scenes, name)(**kw)
    per_step_s = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    shared = args.sampling == "shared"
    for _ in range(args.warmup):
        cpu_baseline(sc, spp, bounces, target_s=min(per_step_s, 3.0), shared=shared)
    vals = []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(sc, spp, bounces, target_s=per_step_s, shared=shared)
        vals.append(last["value"])
    v = float(np.mean(vals))
    if name == "batch_objects":
        config = {"workload": args.workload, "spp": spp, "bounces": bounces, "sampling": args.sampling}
    else:
        ee = args.early_escape if args.early_escape is not None else DEFAULT_EARLY_ESCAPE
        config = single_config(args, sc.H, sc.W, sc.K, sc.C, spp, bounces, n_iter, ee, world)
    line = {"impl": "reference", "metric": "IRT-PS Mrays/s", "value": v, "unit": "Mrays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": dict(last, value=v),
            "e2e": {"value": v, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batch(args):
    """The batched pattern: the objects of the job in one batch per rank (a cost-balanced split of
    the objects over the ranks; one gather of the results at the end), against per-object
    contexts."""
    import torch
    import scenes
    from paper_1811_02357_gb300 import build
    build.build()
    from paper_1811_02357_gb300 import irtps

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _, kw, _, _, n_iter, rspp, rb = WORKLOADS[args.workload]
    job = scenes.batch_objects(seed=4, **kw)  # the same job on every rank
    costs = [float(sc.H * sc.W * sc.K * s_ * b_) for sc, s_, b_ in job]
    parts = split_objects(costs, world)
    mine = parts[rank]
    objs = [job[i] for i in mine]
    stream = torch.cuda.Stream(device=dev)
    img_dtype = irtps.IRTPS_F16 if args.images == "f16" else irtps.IRTPS_F32
    ctxs, imgs = [], []
    opt = irtps.irtps_default_options()
    opt.sampling = 1 if args.sampling == "shared" else 0
    if args.early_escape is not None:
        opt.early_escape = args.early_escape
    for g, (sc, _, _) in zip(mine, objs):
        c = irtps.Context(sc.H, sc.W, sc.lights, sc.env, opt)
        c.set_stream(stream.cuda_stream)
        c.set_state(sc.depth, sc.normals, sc.albedo)
        A = torch.empty((sc.K, sc.C, sc.H, sc.W), dtype=torch.float32, device=dev)
        c.render(rspp, rb, 1000 + g, 0.002, out=A)
        ctxs.append(c)
        imgs.append(A.half() if args.images == "f16" else A)
    torch.cuda.synchronize()
    spp = [o[1] for o in objs]
    bnc = [o[2] for o in objs]
    seed = 1
    # pinned host images and results of the end-to-end path (copied in and out every step)
    host = []
    for a in imgs:
        h = torch.empty(a.shape, dtype=a.dtype, pin_memory=True)
        h.copy_(a.cpu())
        host.append(h)
    outs = [torch.empty((sc.H, sc.W), pin_memory=True) for sc, _, _ in objs]

    def make_batch(use_graph):
        b = irtps.Batch(ctxs, use_graph=use_graph)
        b.set_stream(stream.cuda_stream)
        for c, g in zip(ctxs, mine):  # each object keeps its index in the whole job (its Philox key)
            c.set_object(g)
        return b

    # stage events need the enqueued form; the captured (graph) form is timed once after it
    batch = make_batch(False)
    P = sum(sc.H * sc.W for sc, _, _ in objs)

    def set_all(src, on_device):
        ptrs = (irtps.ctypes.c_void_p * len(src))(*[a.data_ptr() for a in src])
        irtps._check_batch(batch.b, irtps._lib.irtps_batch_set_images(batch.b, ptrs, img_dtype, on_device))
        return batch.stats()

    def step(ev=None):
        """One user step: images in from pinned host memory (iteration 0 of every object), the IRT
        iteration, every object's depth back; ev = four events (start, iteration start / end, end)."""
        if ev:
            ev[0].record(stream)
        s0 = set_all(host, 0)
        if ev:
            ev[1].record(stream)
        batch.iterate(n_iter, spp, bnc, seed)
        if ev:
            ev[2].record(stream)
        st = dict(batch.stats())
        for c, o in zip(ctxs, outs):
            irtps._check(c.h, irtps._lib.irtps_get_depth(c.h, irtps._addr(o.data_ptr()), 0))
        if ev:
            ev[3].record(stream)
        st["set_ps_ms"], st["set_depth_ms"] = s0["ps_ms"], s0["depth_ms"]
        return st

    def per_object():
        segs = 0
        for c, g, a, s_, b_ in zip(ctxs, mine, imgs, spp, bnc):
            c.set_object(g)
            c.set_images(a, dtype=img_dtype, on_device=True)
            c.iterate(n_iter, s_, b_, seed)
            segs += c.stats()["segments"]
        return segs

    def timed(fn, steps):
        out = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            out.append((e0.elapsed_time(e1), r))
        return out

    # the tuner picks the trace grid and pyramid depth (no result bit depends on them)
    if not args.no_autotune and not args.workload.endswith("_profile"):  # profile cases keep the defaults
        set_all(imgs, 1)
        batch.autotune([max(1, s_ // (4 if args.sampling == "shared" else 16)) for s_ in spp], bnc, seed)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = batch.stats()["launches"] + sum(c.stats()["launches"] for c in ctxs)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    res = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            res.append(step(evs[i]))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    launches = batch.stats()["launches"] + sum(c.stats()["launches"] for c in ctxs) - launches0
    ms = sum(e[1].elapsed_time(e[2]) for e in evs)
    ms_e2e = sum(e[0].elapsed_time(e[3]) for e in evs)
    segs = sum(r["segments"] for r in res)
    draws = sum(r["draws"] for r in res)
    nodes = sum(r["node_visits"] for r in res)
    tris = sum(r["tri_tests"] for r in res)
    trace_ms = sum(r["trace_ms"] for r in res)
    primary = sum(r["primary_segments"] for r in res)
    ms_all, segs_all = combine_ranks(ms, segs, world, dev)
    ms_e2e_all, _ = combine_ranks(ms_e2e, segs, world, dev)
    P_all = sum(sc.H * sc.W for sc, _, _ in job)
    value = segs_all / (ms_all / 1e3) / 1e6
    # the results of the job: one gather of every object's surface to rank 0 (outside the timed region)
    sizes = [sc.H * sc.W for sc, _, _ in job]
    local_depth = {g: o.numpy() for g, o in zip(mine, outs)}
    gathered = gather_objects(local_depth, sizes, parts, world, rank, dev)
    # the same step with the iteration replayed as a CUDA graph
    tuning = batch.tuning()
    batch.close()
    batch = make_batch(True)
    batch.set_tuning(*tuning)
    set_all(imgs, 1)
    batch.iterate(n_iter, spp, bnc, seed)
    graph_ms = timed(lambda: (set_all(imgs, 1), batch.iterate(n_iter, spp, bnc, seed)), 1)[0][0]
    # the same job as per-object launches with the batch's options (one context after another)
    per_object()
    po = timed(per_object, max(1, min(2, args.steps)))
    po_ms = sum(r[0] for r in po)
    po_value = sum(r[1] for r in po) / (po_ms / 1e3) / 1e6
    # the plain form: per-object contexts, FP32 images, per-light sampling (the form the
    # mixed-precision batch is compared with); timed when the batch's options differ from it
    plain = None
    if args.images != "f32" or args.sampling != "per_light":
        popt = irtps.irtps_default_options()
        if args.early_escape is not None:
            popt.early_escape = args.early_escape
        pctx = []
        for g, (sc, _, _) in zip(mine, objs):
            c = irtps.Context(sc.H, sc.W, sc.lights, sc.env, popt)
            c.set_stream(stream.cuda_stream)
            c.set_object(g)
            pctx.append(c)
        imgs32 = [a.float() if a.dtype != torch.float32 else a for a in imgs]

        def plain_step():
            for c, a, s_, b_ in zip(pctx, imgs32, spp, bnc):
                c.set_images(a, dtype=irtps.IRTPS_F32, on_device=True)
                c.iterate(n_iter, s_, b_, seed)
            return 0
        plain_step()
        pl_ms = timed(plain_step, 1)[0][0]
        plain = {"pixel_iters_per_s": P * n_iter / (pl_ms / 1e3), "ms_per_step": pl_ms,
                 "what": "the same objects as per-object contexts of the plain form: FP32 images, per-light "
                         "sampling, default options"}
        for c in pctx:
            c.close()
        del imgs32
    e2e = {"value": segs_all / (ms_e2e_all / 1e3) / 1e6, "unit": "Mrays/s",
           "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in host),
           "d2h_bytes_per_step": sum(o.numel() * 4 for o in outs), "steps": args.steps,
           "ms_per_step": ms_e2e_all / args.steps,
           "how": "CUDA events around irtps_batch_set_images (pinned host images; iteration 0), "
                  "irtps_batch_iterate and every object's depth read back, every timed step"}
    clocks = clk.summary()
    mhz = clocks["sm_max_mhz"] or sm_max_mhz()
    ops = OPS_PER_DRAW * draws + OPS_PER_NODE * nodes + OPS_PER_TRI * tris
    achieved = ops / (trace_ms / 1e3) / 1e12
    peak = sm_count(dev) * LANES_PER_SM * mhz * 1e6 / 1e12
    bps, cut = tuning
    line = {"metric": "IRT-PS Mrays/s", "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "objects": len(job), "pixels": P_all,
                       "sides": [sc.H for sc, _, _ in job], "K": [sc.K for sc, _, _ in job],
                       "spp": [o[1] for o in job], "bounces": [o[2] for o in job], "images": args.images,
                       "sampling": args.sampling, "irt_iterations_per_step": n_iter,
                       "trace_blocks_per_sm": bps, "mip_cut": cut,
                       "parallelism": f"objects split over {world} rank(s) by cost" if world > 1 else "one batch",
                       "rank_objects": [len(p) for p in parts],
                       "l2": "inputs larger than L2 (images of all objects, copied in every step)"},
            "pixel_iters_per_s": P_all * n_iter * args.steps / (ms_all / 1e3),
            "primary_mrays_per_s": combine_ranks(0.0, primary, world, dev)[1] / (ms_all / 1e3) / 1e6,
            "per_object_launches": {"value": po_value, "unit": "Mrays/s", "ms_per_step": po_ms / len(po),
                                    "rank": 0 if world > 1 else None},
            "plain_fp32_per_object": plain,
            "speedup_vs_plain_fp32_per_object": (None if plain is None else
                                                 (P * n_iter * args.steps / (ms / 1e3)) / plain["pixel_iters_per_s"]),
            "graph_ms_per_step": graph_ms,
            "speedup_vs_per_object": (segs / (ms / 1e3) / 1e6) / po_value,
            "stage_ms_per_step": {"trace": trace_ms / args.steps,
                                  "ps": sum(r["ps_ms"] for r in res) / args.steps,
                                  "depth": sum(r["depth_ms"] for r in res) / args.steps,
                                  "iteration0_ps": sum(r["set_ps_ms"] for r in res) / args.steps,
                                  "iteration0_depth": sum(r["set_depth_ms"] for r in res) / args.steps},
            "gpu_launches": launches, "clocks": clocks,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_trace (batched)",
                         "launch_ms": trace_ms / (args.steps * n_iter)},
            "e2e": e2e}
    if rank == 0:
        line["gathered_objects"] = len(gathered)
    if rank == 0 and not args.no_accuracy:
        # every context has run set_images and n_iter iterations (the per-object runs were last)
        line["accuracy"] = batch_accuracy(irtps, batch, ctxs, mine, objs, host, spp, bnc, seed,
                                          args.sampling == "shared", n_iter)
    if rank == 0 and not args.no_cpu_baseline:
        sc0, s0, b0 = job[0]
        line["cpu_baseline"] = cpu_baseline(sc0, s0, b0, shared=args.sampling == "shared")
    batch.close()
    for c in ctxs:
        c.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def batch_accuracy(irtps, batch, ctxs, mine, objs, host, spp, bnc, seed, shared, t, n_check=4, n_samples=64):
    """Stage-wise errors of one batched iteration (iteration index t of every object) against the FP64
    oracle for a few of the batch's objects (the largest, the smallest and two between), from each
    object's own GPU state: the oracle
    traces sampled pixels with the object's Philox key and iteration index, solves their normals from
    the same images, and integrates the object's GPU normals exactly (outside the timed region)."""
    import oracle
    order = sorted(range(len(objs)), key=lambda i: objs[i][0].H * objs[i][0].W)
    pick = sorted({order[0], order[-1], order[len(order) // 3], order[2 * len(order) // 3]})[:n_check]
    before = {i: (ctxs[i].depth(), ctxs[i].normals(), ctxs[i].albedo()) for i in pick}
    batch.iterate(1, spp, bnc, seed)
    rng = np.random.default_rng(13)
    errs, derr, lrel = [], [], []
    for i in pick:
        sc = objs[i][0]
        c = ctxs[i]
        K, C, H, W = sc.K, sc.C, sc.H, sc.W
        d_t, n_t, a_t = before[i]
        n_1, d_1 = c.normals(), c.depth()
        lb = c.indirect().reshape(K, C, -1)
        pix = np.sort(rng.choice(H * W, min(n_samples, H * W), replace=False)).astype(np.int32)
        lb_or, _, _ = oracle.trace(d_t, n_t[..., :3], a_t, sc.lights, sc.env, spp[i], bnc[i], seed, t,
                                   pixels=pix, obj=mine[i], shared=shared)
        img = host[i].reshape(K, C, -1)[:, :, pix].float().numpy()[..., None]
        n_or, _, _ = oracle.ps_step(img, a_t.reshape(C, -1)[:, pix], lb_or, sc.lights)
        errs.append(oracle.angular_error_deg(n_1.reshape(-1, 4)[pix, :3], n_or))
        want_d = oracle.poisson_solve(n_1[..., :3].astype(np.float64), 1.0 / W)
        derr.append(float(np.abs(d_1 - want_d).max() / np.ptp(want_d)))
        got = lb[:, :, pix]
        lrel.append(float((np.abs(got - lb_or) / np.maximum(np.abs(lb_or), 1e-30))[np.abs(lb_or) > 1e-6].max()))
    e = np.concatenate(errs)
    return {"objects": [int(mine[i]) for i in pick], "pixels_per_object": n_samples,
            "normal_mean_deg": float(e.mean()), "normal_max_deg": float(e.max()),
            "depth_max_rel_range": max(derr), "lbar_max_rel": max(lrel),
            "how": "per object: the GPU's state before one batched iteration in; the oracle traces sampled pixels "
                   "(same Philox key and iteration, same sampling), solves their normals from the same images, "
                   "and solves the depth of the GPU's normals exactly"}


def sm_count(dev):
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count


def accuracy(oracle, ctx, sc, A_host, spp, bounces, seed, t, n_samples=256, rng_seed=11):
    """Stage-wise errors of one IRT iteration against the FP64 oracle, given the GPU's own
    iteration-t state (outside the timed region).  The GPU runs iteration t; on a sample of
    pixels the oracle traces the same paths over the GPU's surface (Lbar), solves the normals
    from the same (FP16) images with its own Lbar and with the GPU's, and integrates the GPU's
    normals over the whole grid."""
    import torch
    K, C, H, W = sc.K, sc.C, sc.H, sc.W
    d_t, n_t, a_t = ctx.depth(), ctx.normals(), ctx.albedo()
    ctx.iterate(1, spp, bounces, seed)
    n_1, d_1, a_1, v_1 = ctx.normals(), ctx.depth(), ctx.albedo(), ctx.valid()
    rng = np.random.default_rng(rng_seed)
    pix = np.sort(rng.choice(H * W, n_samples, replace=False)).astype(np.int32)
    lb = torch.empty((K, C, H, W), dtype=torch.float32, device="cuda")
    ctx.indirect(out=lb)
    torch.cuda.synchronize()
    lb_gpu = lb.reshape(K, C, -1)[:, :, torch.as_tensor(pix, device="cuda").long()].cpu().numpy()
    del lb
    t0 = time.perf_counter()
    lb_or, _, _ = oracle.trace(d_t, n_t[..., :3], a_t, sc.lights, sc.env, spp, bounces, seed, t, pixels=pix)
    trace_s = time.perf_counter() - t0
    img = A_host.reshape(K, C, -1)[:, :, pix].float().numpy()[..., None]   # (K, C, n, 1)
    rho_t = a_t.reshape(C, -1)[:, pix]
    n_or, rho_or, ok_or = oracle.ps_step(img, rho_t, lb_or, sc.lights)
    n_st, rho_st, ok_st = oracle.ps_step(img, rho_t, lb_gpu.astype(np.float64), sc.lights)
    got_n = n_1.reshape(-1, 4)[pix, :3]
    got_rho = a_1.reshape(C, -1)[:, pix]
    err = oracle.angular_error_deg(got_n, n_or)
    err_st = oracle.angular_error_deg(got_n, n_st)
    want_d = oracle.poisson_solve(n_1[..., :3].astype(np.float64), 1.0 / W)
    rel = np.abs(lb_gpu - lb_or) / np.maximum(np.abs(lb_or), 1e-30)
    return {"iteration": t, "pixels": int(n_samples),
            "normal_mean_deg": float(err.mean()), "normal_max_deg": float(err.max()),
            "albedo_mean_abs": float(np.abs(got_rho - rho_or).mean()),
            "albedo_max_abs": float(np.abs(got_rho - rho_or).max()),
            "depth_max_rel_range": float(np.abs(d_1 - want_d).max() / np.ptp(want_d)),
            "lbar_max_rel": float(rel[np.abs(lb_or) > 1e-6].max()),
            "ps_stage_normal_max_deg": float(err_st.max()),
            "ps_stage_masks_equal": bool(np.array_equal(ok_st, v_1.reshape(-1)[pix].astype(bool))),
            "oracle_trace_s": trace_s,
            "how": "the GPU's iteration-t state (depth, normals, albedo) in; the oracle traces the "
                   "sampled pixels with the same Philox stream, subtracts and solves from the same "
                   "images (normal_*: its own Lbar; ps_stage_*: the GPU's Lbar), and solves the depth "
                   "of the GPU's normals exactly over the whole grid"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bumps_2048", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-e2e", action="store_true",
                    help="batch workloads: leave out the end-to-end run (single objects time it in every step)")
    ap.add_argument("--images", default=None, choices=["f32", "f16"],
                    help="storage type of the input images (default: the workload's; f16 is the "
                         "mixed-precision pattern)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default trace grid and pyramid depth (profiler captures)")
    ap.add_argument("--evaluate", action="store_true",
                    help="also report Table-1-style errors against the ground truth: classic PS and IRT-PS "
                         "with 1, 2 and 3 traced reflections (outside the timed region)")
    ap.add_argument("--sampling", default="per_light", choices=["per_light", "shared"],
                    help="trace sampling: spp paths per (pixel, light), or per pixel for all lights")
    ap.add_argument("--early-escape", type=int, choices=[0, 1], default=None,
                    help="horizon bounds before each trace (default: the library's option default)")
    args = ap.parse_args()
    if args.images is None:
        args.images = WORKLOAD_IMAGES.get(args.workload, "f32")
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOADS[args.workload][0] == "batch_objects":
        return run_batch(args)

    import torch
    import scenes
    from paper_1811_02357_gb300 import build
    build.build()
    from paper_1811_02357_gb300 import irtps

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name, kw, spp, bounces, n_iter, rspp, rb = WORKLOADS[args.workload]
    sc = getattr(scenes, name)(**kw)
    H, W, K, C = sc.H, sc.W, sc.K, sc.C
    seed = 1 + rank
    stream = torch.cuda.Stream(device=dev)
    opt = irtps.irtps_default_options()
    opt.sampling = 1 if args.sampling == "shared" else 0
    for key, val in WORKLOAD_OPTIONS.get(args.workload, {}).items():
        setattr(opt, key, val)
    if args.early_escape is not None:
        opt.early_escape = args.early_escape
    ctx = irtps.Context(H, W, sc.lights, sc.env, opt)
    ctx.set_stream(stream.cuda_stream)
    A0 = torch.empty((K, C, H, W), dtype=torch.float32, device=dev)
    ctx.set_state(sc.depth, sc.normals, sc.albedo)
    ctx.render(rspp, rb, 1000 + rank, 0.002, out=A0)
    torch.cuda.synchronize()
    img_dtype = irtps.IRTPS_F16 if args.images == "f16" else irtps.IRTPS_F32
    A0_in = A0.half() if args.images == "f16" else A0
    del A0
    # the step's inputs and outputs in pinned host memory (the end-to-end path copies them every step)
    A_host = torch.empty((K, C, H, W), dtype=A0_in.dtype, pin_memory=True)
    A_host.copy_(A0_in.cpu())
    outs = {"depth": torch.empty((H, W), pin_memory=True), "normals": torch.empty((H, W, 4), pin_memory=True),
            "albedo": torch.empty((C, H, W), pin_memory=True)}
    in_bytes = A_host.numel() * A_host.element_size()
    big = in_bytes > 256 * 1024 * 1024
    # below twice the L2 size a 512 MB write flushes L2 between timed steps
    flush = None if big else torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lib = irtps._lib

    # the tuner picks the trace grid and pyramid depth (no result bit depends on them)
    if not args.no_autotune and not args.workload.endswith("_profile"):  # profile cases keep the defaults
        ctx.set_images(A0_in, dtype=img_dtype, on_device=True)
        # probes with a fraction of the samples (at most a quarter when light-shared, whose work items
        # are sample chunks of at least 16: fewer samples would change the items the grid shares)
        div = 4 if args.sampling == "shared" else WORKLOAD_TUNE_DIV.get(args.workload, 16)
        ctx.autotune(max(1, spp // div), bounces, seed)
    tuning = ctx.tuning()

    def step(ev=None):
        """One user step through the C ABI; ev = four events (start, iteration start / end, end)."""
        if ev:
            ev[0].record(stream)
        irtps._check(ctx.h, lib.irtps_set_images(ctx.h, irtps._addr(A_host.data_ptr()), img_dtype, 0))
        if ev:
            ev[1].record(stream)
        irtps._check(ctx.h, lib.irtps_iterate(ctx.h, n_iter, spp, bounces, seed, None))
        if ev:
            ev[2].record(stream)
        st = ctx.stats()
        irtps._check(ctx.h, lib.irtps_get_depth(ctx.h, irtps._addr(outs["depth"].data_ptr()), 0))
        irtps._check(ctx.h, lib.irtps_get_normals(ctx.h, irtps._addr(outs["normals"].data_ptr()), 0))
        irtps._check(ctx.h, lib.irtps_get_albedo(ctx.h, irtps._addr(outs["albedo"].data_ptr()), 0))
        if ev:
            ev[3].record(stream)
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = ctx.stats()["launches"]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    tot = dict(segments=0, primary=0, draws=0, nodes=0, tris=0, trace_ms=0.0, ps_ms=0.0, depth_ms=0.0,
               fill_ms=0.0, cg_iters=0, launches=0)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            if flush is not None:
                with torch.cuda.stream(stream):
                    flush.zero_()
            st = step(evs[i])
            tot["segments"] += st["segments"]
            tot["primary"] += st["primary_segments"]
            tot["draws"] += st["draws"]
            tot["nodes"] += st["node_visits"]
            tot["tris"] += st["tri_tests"]
            tot["trace_ms"] += st["trace_ms"]
            tot["ps_ms"] += st["ps_ms"]
            tot["depth_ms"] += st["depth_ms"]
            tot["fill_ms"] += st["fill_ms"]
            tot["cg_iters"] += st["cg_iterations"]
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    launches = ctx.stats()["launches"] - launches0
    ms = sum(e[1].elapsed_time(e[2]) for e in evs)
    ms_e2e = sum(e[0].elapsed_time(e[3]) for e in evs)
    ms_all, segs_all = combine_ranks(ms, tot["segments"], world, dev)
    ms_e2e_all, _ = combine_ranks(ms_e2e, tot["segments"], world, dev)
    value = segs_all / (ms_all / 1e3) / 1e6
    P = H * W
    e2e = {"value": segs_all / (ms_e2e_all / 1e3) / 1e6, "unit": "Mrays/s", "h2d_bytes_per_step": in_bytes,
           "d2h_bytes_per_step": sum(t.numel() * 4 for t in outs.values()), "steps": args.steps,
           "ms_per_step": ms_e2e_all / args.steps,
           "how": "CUDA events around irtps_set_images (pinned host images; runs iteration 0), "
                  "irtps_iterate and the depth / normals / albedo read-back, every timed step"}

    # roofline of the dominant kernel (the trace): algorithmic lane-ops / its event-timed duration
    clocks = clk.summary()
    mhz = clocks["sm_max_mhz"] or sm_max_mhz()
    sms = sm_count(dev)
    ops = OPS_PER_DRAW * tot["draws"] + OPS_PER_NODE * tot["nodes"] + OPS_PER_TRI * tot["tris"]
    trace_launches = args.steps * n_iter
    achieved = ops / (tot["trace_ms"] / 1e3) / 1e12
    peak = sms * LANES_PER_SM * mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": TRACE_DRAM_BYTES.get((args.workload, args.sampling)),
                "kernel": "k_trace",
                "launch_ms": tot["trace_ms"] / trace_launches,
                "note": f"lane-operation issue peak = {sms} SMs x {LANES_PER_SM} lanes x max SM clock; ops "
                        "counted per sampled direction, pyramid node visit and triangle test"}

    line = {"metric": "IRT-PS Mrays/s", "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": single_config(args, H, W, K, C, spp, bounces, n_iter, opt.early_escape, world),
            "tuning": {"trace_blocks_per_sm": tuning[0], "mip_cut": tuning[1]},
            "pixel_iters_per_s": P * n_iter * world * args.steps / (ms_all / 1e3),
            "primary_mrays_per_s": tot["primary"] * world / (ms_all / 1e3) / 1e6,
            "stage_ms_per_step": {"trace": tot["trace_ms"] / args.steps, "ps": tot["ps_ms"] / args.steps,
                                  "depth": tot["depth_ms"] / args.steps, "hole_fill": tot["fill_ms"] / args.steps},
            "cg_iterations_last_solve": tot["cg_iters"] / args.steps,
            "work_per_segment": {"node_visits": tot["nodes"] / max(1, tot["segments"]),
                                 "tri_tests": tot["tris"] / max(1, tot["segments"]),
                                 "draws": tot["draws"] / max(1, tot["segments"])},
            "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "e2e": e2e}
    if rank == 0 and not args.no_accuracy and opt.sampling == 0 and not opt.fill_holes:
        import oracle
        line["accuracy"] = accuracy(oracle, ctx, sc, A_host, spp, bounces, seed, n_iter)
    if args.evaluate:
        line["evaluation"] = evaluate(irtps, sc, spp, n_iter, seed, opt, stream, dev, render_spp=max(spp, rspp))
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, spp, bounces, shared=args.sampling == "shared", single_thread=True)
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
