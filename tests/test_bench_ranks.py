"""Ranks of bench.py on CPU (gloo, world size 2): the whole-job time is the slowest
rank's, the units are summed over ranks, and the reference arm prints from rank 0
only (the other ranks exit without work).  A batch job split over ranks: the
cost-balanced split covers every object once, and one gather of the per-object
results at the end gives rank 0 exactly what a single rank computes alone (the
per-object work here is the oracle's classic PS and integration, iteration 0 of
the loop, on small objects of the batch recipe)."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.combine_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1), world, "cpu")
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_combine_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for _, ms, units in got:
        assert ms == 150.0 and units == 3000.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(12.5, 7, 1, "cpu") == (12.5, 7.0)


def test_reference_arm_prints_on_rank_0_only(tmp_path):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "bowl_64", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "bowl_64", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_split_objects_covers_and_balances():
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    import scenes
    job = scenes.batch_spec()
    costs = [float(side * side * K * spp * b) for _, side, K, spp, b in job]
    for world in (1, 2, 3, 4, 8):
        parts = bench.split_objects(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy largest-first: no rank exceeds the mean by more than the largest object
        assert max(loads) <= sum(costs) / world + max(costs)
        assert all(p == sorted(p) for p in parts)
    assert bench.split_objects(costs, 1) == [list(range(len(costs)))]


def _objects():
    import scenes
    return [scenes.mixed(300 + i, 10 + (7 * i) % 13, 9 + (5 * i) % 11, K=4, C=3) for i in range(7)]


def _work(oracle_mod, sc, i):
    """Iteration 0 of object i: classic PS of its images, integrated (the per-object result)."""
    import numpy as np
    A0 = oracle_mod.render(sc.depth, sc.normals, sc.albedo, sc.lights, sc.env, 4, 1, 10 + i, 0.002)
    hist = oracle_mod.irtps_run(A0, sc.lights, sc.env, 0, 1, 1, 1)
    return hist[0]["depth"].astype(np.float32)


def _split_rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    objs = _objects()
    costs = [float(sc.H * sc.W * sc.K) for sc in objs]
    parts = bench.split_objects(costs, world)
    local = {i: _work(oracle, objs[i], i) for i in parts[rank]}
    got = bench.gather_objects(local, [sc.H * sc.W for sc in objs], parts, world, rank, "cpu")
    q.put((rank, parts, None if got is None else {i: v.tolist() for i, v in got.items()}))
    dist.destroy_process_group()


def test_split_batch_gather_matches_single_rank_gloo():
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in range(2)), key=lambda x: x[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (_, parts0, res0), (_, parts1, res1) = got
    assert parts0 == parts1 and res1 is None
    assert set(parts0[0]).isdisjoint(parts0[1]) and parts0[0] and parts0[1]  # both ranks work
    objs = _objects()
    single = bench.gather_objects({i: _work(oracle, sc, i) for i, sc in enumerate(objs)},
                                  [sc.H * sc.W for sc in objs], [list(range(len(objs)))], 1, 0, "cpu")
    assert sorted(res0) == list(range(len(objs)))
    for i, sc in enumerate(objs):
        assert np.array_equal(np.asarray(res0[i], np.float32), single[i])
        assert single[i].size == sc.H * sc.W
