"""IRT-PS benchmark: Mrays/s of the whole loop on one seeded synthetic workload.

Workload `bumps_512` (default): 512x512 RGB heightfield of 20 Gaussian bumps and
dents plus a 90-degree V-groove, Voronoi albedo, 32x64 RGB cosine environment,
K = 12 lights; trace 256 spp, 2 bounces; one step = one whole job: iteration 0
(classic PS + integration) from device-resident images, then 5 IRT iterations
(pyramid, trace, subtract + PS, integration, D_H).  Input images are rendered
once on the GPU from the ground truth (256 spp, 2 bounces, sigma 0.002).

value      = traced segments (primary, bounce and shadow rays) / second, all ranks
e2e        = the same through the C ABI from pinned host images, results copied back
roofline   = the trace kernel (dominant): algorithmic lane operations per second
             against the lane-issue peak (bound "alu")
cpu_baseline = the oracle (plain C++) on the host cores over a pixel sample
evaluation (--evaluate) = errors against the ground truth (height, albedo, normal; the paper's
             evaluation measures) of classic PS and of IRT-PS with 1, 2 and 3 traced reflections

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
    # name: (scene factory, its arguments, spp, bounces, IRT iterations per job, render spp, render bounces)
    "bumps_512": ("bumps_512", {}, 256, 2, 5, 256, 2),
    "bowl_64": ("bowl_64", {}, 64, 1, 3, 256, 1),
    # a small case of the same kernels for profiler captures (one IRT iteration per job)
    "bumps_256_profile": ("bumps_512", {"H": 256, "W": 256}, 32, 2, 1, 32, 2),
    # the 2048x2048, K = 32 configuration at an eighth of its samples (64 spp), one IRT iteration per job
    "bumps_2048_spp64": ("bumps_2048", {}, 64, 2, 1, 4, 1),
    # the 4096x4096, K = 64 configuration at a sixty-fourth of its samples (16 spp), one IRT iteration per job
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

# Algorithmic lane operations per unit of trace work (counted from the formulas:
# Philox4x32-10 = 10 rounds x (2 mul.hi + 2 mul.lo + 4 xor) + 9 x 2 key adds;
# cosine direction = uniforms, 2 sqrt, turn sine/cosine polynomial, Duff basis,
# basis combination; node visit = node bounds, two exit parameters, height at the
# entry, compare; triangle test = Moeller-Trumbore with its four rejections).
OPS_PER_DRAW = 98 + 47
OPS_PER_NODE = 16
OPS_PER_TRI = 57
SM_COUNT = 152
LANES_PER_SM = 128
# DRAM bytes (read + write) of one trace launch of a workload, from the ncu capture summarised in
# profiles/k_trace_bumps512_dram.md (the kernel has not changed since)
TRACE_DRAM_BYTES = {"bumps_512": 19.29e6 + 2.27e6}
# the same for light-shared sampling (profiles/k_trace_shared_bumps512_dram.md)
TRACE_DRAM_BYTES_SHARED = {"bumps_512": 322.63e6 + 270.69e6}


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
    line = {"impl": "reference", "metric": "IRT-PS Mrays/s", "value": v, "unit": "Mrays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "spp": spp, "bounces": bounces, "sampling": args.sampling},
            "cpu_baseline": dict(last, value=v),
            "e2e": {"value": v, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batch(args):
    """The batched pattern: all objects in one batch against per-object contexts."""
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
    _, _, _, _, n_iter, rspp, rb = WORKLOADS[args.workload]
    _, kw, _, _, _, _, _ = WORKLOADS[args.workload]
    objs = scenes.batch_objects(seed=4 + 100 * rank, **kw)
    stream = torch.cuda.Stream(device=dev)
    img_dtype = irtps.IRTPS_F16 if args.images == "f16" else irtps.IRTPS_F32
    ctxs, imgs = [], []
    opt = irtps.irtps_default_options()
    opt.sampling = 1 if args.sampling == "shared" else 0
    if args.early_escape is not None:
        opt.early_escape = args.early_escape
    for i, (sc, _, _) in enumerate(objs):
        c = irtps.Context(sc.H, sc.W, sc.lights, sc.env, opt)
        c.set_stream(stream.cuda_stream)
        c.set_state(sc.depth, sc.normals, sc.albedo)
        A = torch.empty((sc.K, sc.C, sc.H, sc.W), dtype=torch.float32, device=dev)
        c.render(rspp, rb, 1000 + i, 0.002, out=A)
        ctxs.append(c)
        imgs.append(A.half() if args.images == "f16" else A)
    torch.cuda.synchronize()
    spp = [o[1] for o in objs]
    bnc = [o[2] for o in objs]
    seed = 1 + rank
    # stage events need the enqueued form; the captured (graph) form is timed once after it
    batch = irtps.Batch(ctxs, use_graph=False)
    batch.set_stream(stream.cuda_stream)
    P = sum(sc.H * sc.W for sc, _, _ in objs)

    def set_all(host=None):
        src = host if host is not None else imgs
        ptrs = (irtps.ctypes.c_void_p * len(src))(*[a.data_ptr() for a in src])
        irtps._check_batch(batch.b, irtps._lib.irtps_batch_set_images(batch.b, ptrs, img_dtype,
                                                                      0 if host is not None else 1))
        return batch.stats()

    def batched():
        s0 = set_all()
        batch.iterate(n_iter, spp, bnc, seed)
        st = dict(batch.stats())
        for k in ("ps_ms", "depth_ms"):
            st[k] += s0[k]
        return st

    def per_object():
        segs = 0
        for c, s_, b_ in zip(ctxs, spp, bnc):
            c.set_images(imgs[ctxs.index(c)], dtype=img_dtype, on_device=True)
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
        set_all()
        batch.autotune([max(1, s_ // (4 if args.sampling == "shared" else 16)) for s_ in spp], bnc, seed)
    for _ in range(args.warmup):
        batched()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = batch.stats()["launches"] + sum(c.stats()["launches"] for c in ctxs)
    with ClockSampler(local) as clk:
        res = timed(batched, args.steps)
        if world > 1:
            torch.distributed.barrier()
    launches = batch.stats()["launches"] + sum(c.stats()["launches"] for c in ctxs) - launches0
    ms = sum(r[0] for r in res)
    segs = sum(r[1]["segments"] for r in res)
    draws = sum(r[1]["draws"] for r in res)
    nodes = sum(r[1]["node_visits"] for r in res)
    tris = sum(r[1]["tri_tests"] for r in res)
    trace_ms = sum(r[1]["trace_ms"] for r in res)
    primary = sum(r[1]["primary_segments"] for r in res)
    ms_all, segs_all = combine_ranks(ms, segs, world, dev)
    value = segs_all / (ms_all / 1e3) / 1e6
    # the same step with the iteration replayed as a CUDA graph
    tuning = batch.tuning()
    batch.close()
    batch = irtps.Batch(ctxs, use_graph=True)
    batch.set_stream(stream.cuda_stream)
    batch.set_tuning(*tuning)
    batched()
    graph_ms = timed(batched, 1)[0][0]
    # the same job as per-object launches of the plain form (one context after another)
    per_object()
    po = timed(per_object, max(1, min(2, args.steps)))
    po_ms = sum(r[0] for r in po)
    po_value = sum(r[1] for r in po) / (po_ms / 1e3) / 1e6

    e2e = None
    if not args.no_e2e:
        host = []
        for a in imgs:
            h = torch.empty(a.shape, dtype=a.dtype, pin_memory=True)
            h.copy_(a.cpu())
            host.append(h)
        outs = [torch.empty((sc.H, sc.W), pin_memory=True) for sc, _, _ in objs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        set_all(host)
        batch.iterate(n_iter, spp, bnc, seed)
        segs_e2e = batch.stats()["segments"]
        for c, o in zip(ctxs, outs):
            irtps._check(c.h, irtps._lib.irtps_get_depth(c.h, irtps._addr(o.data_ptr()), 0))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": segs_e2e / dt / 1e6, "unit": "Mrays/s",
               "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in host),
               "d2h_bytes_per_step": sum(o.numel() * 4 for o in outs), "steps": 1}
    clocks = clk.summary()
    mhz = clocks["sm_max_mhz"] or sm_max_mhz()
    ops = OPS_PER_DRAW * draws + OPS_PER_NODE * nodes + OPS_PER_TRI * tris
    achieved = ops / (trace_ms / 1e3) / 1e12
    peak = SM_COUNT * LANES_PER_SM * mhz * 1e6 / 1e12
    bps, cut = tuning
    line = {"metric": "IRT-PS Mrays/s", "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "objects": len(objs), "pixels": P,
                       "sides": [sc.H for sc, _, _ in objs], "K": [sc.K for sc, _, _ in objs], "spp": spp,
                       "bounces": bnc, "images": args.images, "sampling": args.sampling,
                       "irt_iterations_per_step": n_iter,
                       "trace_blocks_per_sm": bps, "mip_cut": cut, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (images of all objects)"},
            "pixel_iters_per_s": P * n_iter * world * args.steps / (ms_all / 1e3),
            "primary_mrays_per_s": primary * world / (ms_all / 1e3) / 1e6,
            "per_object_launches": {"value": po_value, "unit": "Mrays/s", "ms_per_step": po_ms / len(po)},
            "graph_ms_per_step": graph_ms,
            "speedup_vs_per_object": value / po_value,
            "stage_ms_per_step": {"trace": trace_ms / args.steps,
                                  "ps": sum(r[1]["ps_ms"] for r in res) / args.steps,
                                  "depth": sum(r[1]["depth_ms"] for r in res) / args.steps},
            "gpu_launches": launches, "clocks": clocks,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_trace (batched)",
                         "launch_ms": trace_ms / (args.steps * n_iter)},
            "e2e": e2e}
    if rank == 0 and not args.no_cpu_baseline:
        sc0, s0, b0 = objs[0]
        line["cpu_baseline"] = cpu_baseline(sc0, s0, b0, shared=args.sampling == "shared")
    batch.close()
    for c in ctxs:
        c.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bumps_512", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--images", default="f32", choices=["f32", "f16"],
                    help="storage type of the input images (f16: the mixed-precision pattern)")
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
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    img_dtype = irtps.IRTPS_F16 if args.images == "f16" else irtps.IRTPS_F32
    A0_in = A0.half() if args.images == "f16" else A0

    def job():
        ctx.set_images(A0_in, dtype=img_dtype, on_device=True)
        ctx.iterate(n_iter, spp, bounces, seed)
        return ctx.stats()

    # the tuner picks the trace grid and pyramid depth (no result bit depends on them)
    if not args.no_autotune and not args.workload.endswith("_profile"):  # profile cases keep the defaults
        ctx.set_images(A0_in, dtype=img_dtype, on_device=True)
        # probes with a sixteenth of the samples (a quarter when light-shared, whose work items are
        # sample chunks of at least 16: fewer samples would change the items the grid shares)
        ctx.autotune(max(1, spp // (4 if args.sampling == "shared" else 16)), bounces, seed)
    tuning = ctx.tuning()

    for _ in range(args.warmup):
        job()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = ctx.stats()["launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    tot = dict(segments=0, primary=0, draws=0, nodes=0, tris=0, trace_ms=0.0, ps_ms=0.0, depth_ms=0.0,
               fill_ms=0.0, cg_iters=0)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[i][0].record(stream)
            st = job()
            ev[i][1].record(stream)
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
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_all, segs_all = combine_ranks(ms, tot["segments"], world, dev)
    value = segs_all / (ms_all / 1e3) / 1e6
    P = H * W

    # end to end through the C ABI: pinned host images in, results back to pinned host memory
    e2e = None
    if not args.no_e2e:
        A0_host = torch.empty((K, C, H, W), dtype=A0_in.dtype, pin_memory=True)
        A0_host.copy_(A0_in.cpu())
        outs = {"depth": torch.empty((H, W), pin_memory=True), "normals": torch.empty((H, W, 4), pin_memory=True),
                "albedo": torch.empty((C, H, W), pin_memory=True)}
        lib = irtps._lib
        steps_e2e = max(1, min(args.steps, 3))
        segs_e2e = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            irtps._check(ctx.h, lib.irtps_set_images(ctx.h, irtps._addr(A0_host.data_ptr()), img_dtype, 0))
            irtps._check(ctx.h, lib.irtps_iterate(ctx.h, n_iter, spp, bounces, seed, None))
            segs_e2e += ctx.stats()["segments"]
            irtps._check(ctx.h, lib.irtps_get_depth(ctx.h, irtps._addr(outs["depth"].data_ptr()), 0))
            irtps._check(ctx.h, lib.irtps_get_normals(ctx.h, irtps._addr(outs["normals"].data_ptr()), 0))
            irtps._check(ctx.h, lib.irtps_get_albedo(ctx.h, irtps._addr(outs["albedo"].data_ptr()), 0))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": segs_e2e / dt / 1e6, "unit": "Mrays/s",
               "h2d_bytes_per_step": A0_host.numel() * A0_host.element_size(),
               "d2h_bytes_per_step": sum(t.numel() * 4 for t in outs.values()), "steps": steps_e2e}

    # roofline of the dominant kernel (the trace): algorithmic lane-ops / its event-timed duration
    clocks = clk.summary()
    mhz = clocks["sm_max_mhz"] or sm_max_mhz()
    ops = OPS_PER_DRAW * tot["draws"] + OPS_PER_NODE * tot["nodes"] + OPS_PER_TRI * tot["tris"]
    trace_launches = args.steps * n_iter
    achieved = ops / (tot["trace_ms"] / 1e3) / 1e12
    peak = SM_COUNT * LANES_PER_SM * mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": (TRACE_DRAM_BYTES if args.sampling == "per_light" else
                            TRACE_DRAM_BYTES_SHARED).get(args.workload),
                "kernel": "k_trace",
                "launch_ms": tot["trace_ms"] / trace_launches,
                "note": "lane-operation issue peak = 152 SMs x 128 lanes x max SM clock; ops counted per "
                        "sampled direction, pyramid node visit and triangle test"}

    line = {"metric": "IRT-PS Mrays/s", "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "H": H, "W": W, "K": K, "C": C, "spp": spp, "images": args.images,
                       "sampling": args.sampling, "trace_blocks_per_sm": tuning[0], "mip_cut": tuning[1],
                       "options": dict(WORKLOAD_OPTIONS.get(args.workload, {}), early_escape=opt.early_escape),
                       "bounces": bounces, "irt_iterations_per_step": n_iter, "parallelism": f"replicas{world}",
                       "l2": "512 MB buffer written between timed steps"},
            "pixel_iters_per_s": P * n_iter * world * args.steps / (ms_all / 1e3),
            "primary_mrays_per_s": tot["primary"] * world / (ms_all / 1e3) / 1e6,
            "stage_ms_per_step": {"trace": tot["trace_ms"] / args.steps, "ps": tot["ps_ms"] / args.steps,
                                  "depth": tot["depth_ms"] / args.steps, "hole_fill": tot["fill_ms"] / args.steps},
            "cg_iterations_last_solve": tot["cg_iters"] / args.steps,
            "work_per_segment": {"node_visits": tot["nodes"] / max(1, tot["segments"]),
                                 "tri_tests": tot["tris"] / max(1, tot["segments"]),
                                 "draws": tot["draws"] / max(1, tot["segments"])},
            "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "e2e": e2e}
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
