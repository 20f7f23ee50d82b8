"""The allocation-free bounding-cube entry point (rpy_bounding_cube_noalloc),
for callers that cannot allocate device memory, against the cube that the
tree builder computes (rpy_tree_build + rpy_tree_export), on two calls in a
row.  This file is collected last on purpose."""
import numpy as np
import pytest

import paper_1711_02976_gb300 as rp

pytestmark = pytest.mark.gpu


def test_bounding_cube_noalloc_matches_tree_cube():
    import torch
    rng = np.random.default_rng(77)
    # the second call is smaller than the first, so stale partials of the
    # first call remain in the shared scratch array and must not be read
    for n, scale, shift in ((300_001, 2.0, -0.5), (5_000, 0.1, 3.0)):
        pos = rng.random((n, 3)) * scale + shift
        P = torch.from_numpy(pos).cuda()
        t = rp.rpy_tree_build(P, n, 1e-3, 3)
        ref = rp.rpy_tree_export(t, "cube")[0]
        cube = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
        rp.rpy_bounding_cube_noalloc(P, n, cube)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(cube.cpu().numpy(), ref)   # same arithmetic: bit-exact
        t.close()


def test_bounding_cube_noalloc_limits():
    import torch
    P = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    cube = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(rp.RpyError) as e:
        rp.rpy_bounding_cube_noalloc(P, 33_554_433, cube)
    assert e.value.status == -1 and "33554432" in str(e.value)
    with pytest.raises(rp.RpyError) as e:
        rp.rpy_bounding_cube_noalloc(P, 0, cube)
    assert e.value.status == -1 and "at least 1" in str(e.value)
    with pytest.raises(rp.RpyError) as e:
        rp.rpy_bounding_cube_noalloc(None, 4, cube)
    assert e.value.status == -1 and "NULL" in str(e.value)
    P[2, 1] = float("nan")
    rp.rpy_bounding_cube_noalloc(P, 4, cube)
    assert np.isnan(cube.cpu().numpy()[3])


def test_bounding_cube_noalloc_allocates_nothing():
    """The entry point's promise: after its first call on the device (the one-time
    lookup of the fixed array's address), a call leaves the device's free memory
    exactly as it was."""
    import torch
    n = 1_000_003
    P = torch.rand((n, 3), dtype=torch.float64, device="cuda")
    cube = torch.empty(4, dtype=torch.float64, device="cuda")
    rp.rpy_bounding_cube_noalloc(P, n, cube)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rp.rpy_bounding_cube_noalloc(P, n, cube)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
