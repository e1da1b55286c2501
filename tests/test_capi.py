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
    assert o.stop_tol == 0.0 and o.precond == 2 and o.use_graph == 0 and o.sampling == 0
    assert o.irls_iters == 0 and abs(o.irls_delta - 0.05) < 1e-8 and o.early_escape == 2 and o.fill_holes == 0


def test_struct_layouts_match_header(binding, tmp_path):
    """Field offsets and sizes of the binding's structs equal those the C compiler gives the header's."""
    import subprocess
    structs = {"irtps_options": binding.irtps_options, "irtps_stats": binding.irtps_stats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "irtps.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)


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
