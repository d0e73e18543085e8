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


def test_noalloc_bad_offset_marks_voxels_nan(mm):
    """An offset beyond n_obs is caught by the kernel's own range check (no
    observation is read through it): the two voxels it bounds report NaN, the
    cost is NaN, every other voxel keeps its value."""
    import torch
    s, pts, po, raw, cen = tiny_scene()
    dev = torch.device("cuda")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    with mm.BundleAdjuster() as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        ref_lam = ba.planes()[:, 0]
    off = s.voxel_off.copy()
    k = 3
    off[k] = s.n_obs + 7  # voxel k-1 ends and voxel k starts out of range
    cost = torch.zeros(1, dtype=torch.float64, device=dev)
    lam = torch.zeros(s.n_voxels, dtype=torch.float64, device=dev)
    mm.ba_eval_cost_noalloc(s.n_scans, T(off), T(s.obs_scan), T(cen), T(s.pose_init), cost, lam)
    torch.cuda.synchronize()
    got = lam.cpu().numpy()
    assert np.isnan(cost.item())
    assert np.isnan(got[k - 1]) and np.isnan(got[k])
    keep = np.ones(s.n_voxels, bool)
    keep[[k - 1, k]] = False
    np.testing.assert_allclose(got[keep], ref_lam[keep], rtol=1e-9, atol=1e-15)


def test_noalloc_on_a_side_stream(mm):
    """The kind of stream a mapping loop runs on: ordered on a torch side
    stream, the result equals the handle path's."""
    import torch
    s, pts, po, raw, cen = tiny_scene()
    dev = torch.device("cuda")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    with mm.BundleAdjuster() as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_gt)
        ref = ba.cost()
        ref_lam = ba.planes()[:, 0]
    inputs = (T(s.voxel_off), T(s.obs_scan), T(cen), T(s.pose_gt))
    cost = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    lam = torch.full((s.n_voxels,), -1.0, dtype=torch.float64, device=dev)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        mm.ba_eval_cost_noalloc(s.n_scans, *inputs, cost, lam, stream=side)
    side.synchronize()
    assert cost.item() == pytest.approx(ref, rel=COST_TOL)
    np.testing.assert_allclose(lam.cpu().numpy(), ref_lam, rtol=1e-9, atol=1e-15)


def test_noalloc_wrapper_refuses_short_or_strided_tensors(mm):
    """The binding checks shapes and contiguity before the call, so nothing is
    written out of bounds and no hidden copy is made."""
    import torch
    s, pts, po, raw, cen = tiny_scene()
    dev = torch.device("cuda")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    vo, os_, ag, P = T(s.voxel_off), T(s.obs_scan), T(cen), T(s.pose_init)
    cost = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        mm.ba_eval_cost_noalloc(s.n_scans, vo, os_, ag, P, cost,
                                torch.zeros(s.n_voxels - 1, dtype=torch.float64, device=dev))
    with pytest.raises(ValueError):
        mm.ba_eval_cost_noalloc(s.n_scans, vo, os_, ag, P, cost,
                                torch.zeros(2 * s.n_voxels, dtype=torch.float64, device=dev)[::2])
    with pytest.raises(ValueError):
        mm.ba_eval_cost_noalloc(s.n_scans, vo, os_, ag[:-1], P, cost)
    with pytest.raises(ValueError):
        mm.ba_eval_cost_noalloc(s.n_scans + 1, vo, os_, ag, P, cost)
