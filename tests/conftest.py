import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def lib():
    """The CUDA library binding; GPU tests fail (not skip) when it cannot run."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1811_02357_gb300 import build
    build.build()
    from paper_1811_02357_gb300 import irtps
    return irtps


def rel_close(got, want, rtol, atol=0.0):
    """|got - want| <= rtol * |want| + atol elementwise; returns (ok, worst ratio)."""
    import numpy as np
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want)
    lim = rtol * np.abs(want) + atol
    return bool(np.all(err <= lim)), float(np.max(err / np.maximum(lim, 1e-300)))
