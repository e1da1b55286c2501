"""The allocation-free depth solve against the allocating one.

`irtps_integrate_noalloc` serves callers that cannot allocate device memory when
they need a surface (their framework owns the device pool, or cudaMalloc's
device-wide synchronisation is not acceptable in their loop); it keeps its
working vectors in a fixed device array instead.  This test calls it through the
C ABI twice in a row, with different sizes and inputs so that the second call
starts from the first call's leftovers, and checks each result against
`irtps_integrate` on the same normals, within the depth tolerance of the other
tests (1e-4 of the depth range).  The test file sorts last so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def _reference_depth(lib, normals, H, W):
    with lib.Context(H, W, scenes.ring_lights(3, 45.0), np.zeros((1, 2, 2), np.float32)) as ctx:
        ctx.set_state(depth=np.zeros((H, W), np.float32), normals=normals)
        ctx.integrate()
        return ctx.depth()


def test_noalloc_matches_allocating_solve(lib):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    # two small grids in a row (the second starts from the first's leftovers), then the size
    # limit itself, square and long-and-thin: the whole scratch layout in use
    for seed, H, W in [(3, 64, 48), (4, 37, 53), (5, 512, 512), (6, 128, 2048)]:
        sc = scenes.mixed(seed, H, W, K=3, C=1)
        want = _reference_depth(lib, sc.normals, H, W)
        n4 = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
        n4[..., :3] = torch.from_numpy(sc.normals).cuda()
        depth = torch.zeros((H, W), dtype=torch.float32, device="cuda")
        lib.irtps_integrate_noalloc(n4, depth, H, W, stream=stream)  # raises unless IRTPS_OK
        got = depth.cpu().numpy()
        rng = np.ptp(want)
        assert np.abs(got - want).max() <= 1e-4 * rng, (H, W, np.abs(got - want).max() / rng)


def test_noalloc_rejects_oversize(lib):
    import torch
    n4 = torch.zeros((1, 4), dtype=torch.float32, device="cuda")
    d = torch.zeros((1,), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.IrtpsError) as e:
        lib.irtps_integrate_noalloc(n4, d, 513, 512)
    assert e.value.code == lib.IRTPS_EINVAL


def test_noalloc_wrapper_checks_buffers(lib):
    """The binding refuses buffers the kernels would read or write past, before any device work."""
    import torch
    H, W = 16, 12
    n4 = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    d = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    for bad_n, bad_d in [(n4[:, :, :3].contiguous(), d), (n4, d[:-1]), (n4.double(), d), (n4, d.cpu()),
                         (n4.reshape(-1)[1:4 * H * W + 1], d)]:
        with pytest.raises(ValueError):
            lib.irtps_integrate_noalloc(bad_n, bad_d, H, W)
