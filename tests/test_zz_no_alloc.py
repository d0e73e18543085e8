"""The allocation-free cost entry point agrees with the handle-based path.

ba_eval_cost_noalloc serves callers that cannot allocate device memory when
they need a cost (an on-vehicle mapping loop with a fixed memory budget, or a
host whose own allocator holds the GPU memory).  It keeps its scratch in a
library-owned device array, so two calls in a row must each give the same
answer as the ordinary path, with nothing left over from the first call.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from tests._util import tiny_scene

pytestmark = pytest.mark.gpu

COST_TOL = 1e-10


@pytest.fixture(scope="module")
def mm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2608_14266_gb300 as mm
    assert torch.cuda.is_available()
    return mm


def test_noalloc_cost_matches_handle_path_twice(mm):
    import torch
    s, pts, po, raw, cen = tiny_scene()
    dev = torch.device("cuda")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    vo, os_, ag = T(s.voxel_off), T(s.obs_scan), T(cen)
    with mm.BundleAdjuster() as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        for poses in (s.pose_init, s.pose_gt):  # two calls in a row, different answers
            ba.set_state(poses)
            ref_cost = ba.cost()
            ref_lam = ba.planes()[:, 0]
            cost = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
            lam = torch.full((s.n_voxels,), -1.0, dtype=torch.float64, device=dev)
            mm.ba_eval_cost_noalloc(s.n_scans, vo, os_, ag, T(poses), cost, lam)
            torch.cuda.synchronize()
            assert cost.item() == pytest.approx(ref_cost, rel=COST_TOL)
            np.testing.assert_allclose(lam.cpu().numpy(), ref_lam, rtol=1e-9, atol=1e-15)


def test_noalloc_limits_and_bad_indices(mm):
    import torch
    from paper_2608_14266_gb300 import _lib
    s, pts, po, raw, cen = tiny_scene()
    dev = torch.device("cuda")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    cost = torch.zeros(1, dtype=torch.float64, device=dev)
    # beyond the stated maximum: rejected before any GPU work
    st = _lib.lib().ba_eval_cost_noalloc(s.n_scans, _lib.BA_NOALLOC_MAX_VOXELS + 1, _lib.BA_NOALLOC_MAX_VOXELS + 1,
                                         1, 1, 1, 1, cost.data_ptr(), None, None)
    assert st == 7  # BA_ERR_CAPACITY
    # an out-of-range scan index is caught by the kernel's own bounds check
    bad = s.obs_scan.copy()
    bad[5] = s.n_scans + 3
    mm.ba_eval_cost_noalloc(s.n_scans, T(s.voxel_off), T(bad), T(cen), T(s.pose_init), cost)
    torch.cuda.synchronize()
    assert np.isnan(cost.item())
    # and the next good call is not affected by the previous one's error
    with mm.BundleAdjuster() as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        ref = ba.cost()
    mm.ba_eval_cost_noalloc(s.n_scans, T(s.voxel_off), T(s.obs_scan), T(cen), T(s.pose_init), cost)
    torch.cuda.synchronize()
    assert cost.item() == pytest.approx(ref, rel=COST_TOL)
