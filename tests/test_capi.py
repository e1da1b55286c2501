"""The C-ABI library builds, loads and exports every entry point of include/irtps.h;
argument validation runs on the host (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "irtps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(irtps_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def binding():
    from paper_1811_02357_gb300 import build
    build.build()
    from paper_1811_02357_gb300 import irtps
    return irtps


def test_every_declared_symbol_is_exported(binding):
    names = _declared()
    assert len(names) >= 20
    lib = ctypes.CDLL(binding.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(binding.EXPORTED) == names


def test_default_options(binding):
    o = binding.irtps_default_options()
    assert o.shadow_rays == 1 and abs(o.tau_lo - 0.02) < 1e-8 and abs(o.tau_hi - 0.98) < 1e-7
    assert o.cond_max == 1e8 and abs(o.nz_min - 0.05) < 1e-8 and o.cg_tol == 1e-9
    assert o.stop_tol == 0.0 and o.precond == 1


def test_struct_layouts_match_header(binding):
    # sizes of the option / stats structs as the C compiler lays them out
    assert ctypes.sizeof(binding.irtps_options) == 64
    assert ctypes.sizeof(binding.irtps_stats) == 8 * 3 + 8 + 8 * 3 + 8 + 8 * 2 + 8 * 3 + 8 + 8


@pytest.mark.parametrize("args,needle", [
    (dict(H=1, W=8, K=4, C=1), "H, W >= 2"),
    (dict(H=8, W=8, K=2, C=1), "3 <= K"),
    (dict(H=8, W=8, K=65, C=1), "3 <= K"),
    (dict(H=8, W=8, K=4, C=2), "C in {1,3}"),
])
def test_create_rejects_bad_sizes(binding, args, needle):
    lights = scenes.ring_lights(max(args["K"], 1), 45.0)
    with pytest.raises(binding.IrtpsError) as e:
        binding.irtps_create(args["H"], args["W"], args["K"], args["C"], lights, np.zeros((1, 2, 2)))
    assert e.value.code == binding.IRTPS_EINVAL and needle in str(e.value)


def test_create_rejects_coplanar_lights(binding):
    lights = np.array([[1, 0, 1], [-1, 0, 1], [0.5, 0, 1], [-0.5, 0, 1]], np.float32)
    lights /= np.linalg.norm(lights, axis=1, keepdims=True)
    with pytest.raises(binding.IrtpsError) as e:
        binding.irtps_create(8, 8, 4, 1, lights, np.zeros((1, 2, 2)))
    assert e.value.code == binding.IRTPS_EINVAL and "coplanar" in str(e.value)
