"""Host-side parts of bench.py and the workload recipes (no GPU).

* The evaluation errors the benchmark reports equal the oracle's definitions of the
  paper's evaluation measures (height, albedo and normal error), on random estimates.
* The batched workload follows its recipe: 64 objects, sides log-uniform in 96..1024,
  K in {4, 8, 16, 32}, spp in {64, 128, 256}, bounces in {1, 2}.
* The workload table is self-consistent (scene factories, option names, traffic entries,
  image types and tuner divisors).
"""
import json
import os
import sys

import numpy as np

import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_evaluation_errors_match_oracle(oracle_mod):
    sys.path.insert(0, ROOT)
    import bench
    sc = scenes.mixed(12, 21, 17, K=4, C=3)
    rng = np.random.default_rng(3)
    depth = (sc.depth + rng.normal(0, 0.01, sc.depth.shape)).astype(np.float32)
    n = sc.normals + rng.normal(0, 0.05, sc.normals.shape)
    n = (n / np.linalg.norm(n, axis=-1, keepdims=True)).astype(np.float32)
    n4 = np.concatenate([n, np.ones(n.shape[:2] + (1,), np.float32)], axis=-1)
    albedo = (sc.albedo + rng.normal(0, 0.02, sc.albedo.shape)).astype(np.float32)
    got = bench.gt_errors(sc, depth, n4, albedo)
    assert np.isclose(got["height"], oracle_mod.height_error(sc.depth, depth), rtol=1e-12)
    assert np.isclose(got["albedo"], oracle_mod.albedo_error(sc.albedo, albedo), rtol=1e-12)
    assert np.isclose(got["normal"], oracle_mod.normal_error(sc.normals, n), rtol=1e-12)
    ang = oracle_mod.angular_error_deg(sc.normals, n).mean()
    assert np.isclose(got["normal_deg"], ang, rtol=1e-9)


def test_batch_recipe():
    spec = scenes.batch_spec()
    assert len(spec) == 64
    sides = np.array([s[1] for s in spec])
    assert sides.min() >= 96 and sides.max() <= 1024
    assert {s[2] for s in spec} <= {4, 8, 16, 32} and {s[3] for s in spec} <= {64, 128, 256}
    assert {s[4] for s in spec} <= {1, 2}
    # log-uniform: about half of the sides below the geometric mean of the range
    assert 0.3 < (sides < np.sqrt(96 * 1024)).mean() < 0.7
    assert len({s[0] for s in spec}) == 64  # every object its own scene seed


def test_workload_table_is_consistent():
    """Every workload names a scene factory, its options are fields of irtps_options, and
    the traced-roofline traffic table only names workloads that exist."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1811_02357_gb300 import irtps
    fields = {name for name, _ in irtps.irtps_options._fields_}
    for name, (factory, kw, spp, bounces, n_iter, rspp, rb) in bench.WORKLOADS.items():
        assert callable(getattr(scenes, factory)), name
        assert n_iter >= 1 and rspp >= 1 and rb in (1, 2, 3), name
        assert spp is None or (spp >= 1 and bounces in (1, 2, 3)), name
    for name, opts in bench.WORKLOAD_OPTIONS.items():
        assert name in bench.WORKLOADS and set(opts) <= fields, name
    for (name, sampling), traffic in bench.TRACE_DRAM_BYTES.items():
        assert name in bench.WORKLOADS and sampling in ("per_light", "shared") and traffic > 0
    for table in (bench.WORKLOAD_IMAGES, bench.WORKLOAD_TUNE_DIV):
        assert set(table) <= set(bench.WORKLOADS)


def test_reference_arm_config_matches_ours(tmp_path):
    """The reference arm prints the same config as ours for a single-object workload (built by the
    same function from the workload), and its early-escape default is the library's."""
    import argparse
    import subprocess
    sys.path.insert(0, ROOT)
    import bench
    from paper_1811_02357_gb300 import irtps
    assert bench.DEFAULT_EARLY_ESCAPE == irtps.irtps_default_options().early_escape
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "bowl_64", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    import scenes
    sc = scenes.bowl_64()
    _, _, spp, bounces, n_iter, _, _ = bench.WORKLOADS["bowl_64"]
    args = argparse.Namespace(workload="bowl_64", images=bench.WORKLOAD_IMAGES.get("bowl_64", "f32"),
                              sampling="per_light")
    ours = bench.single_config(args, sc.H, sc.W, sc.K, sc.C, spp, bounces, n_iter,
                               irtps.irtps_default_options().early_escape, 1)
    assert line["config"] == json.loads(json.dumps(ours))
