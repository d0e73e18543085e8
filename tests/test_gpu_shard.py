"""A voxel-sharded solve inside the library: one problem's voxels split over
two handles on one GPU, their g, H and cost partials summed on the host (the
all-reduce a multi-GPU run would do), every shard solving and deciding on the
totals.  The shards' poses stay bit-identical, and they follow the unsharded
solve to the precision's rounding (the sums only change order)."""
import numpy as np
import pytest

import oracle
import scenegen
from tests._util import pose_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2608_14266_gb300 as mm
    assert torch.cuda.is_available()
    return mm


def _scene():
    p = scenegen.SceneParams(n_scans=60, n_voxels=6000, obs_min=5, obs_max=20, pts_per_obs=16, noise_sigma=0.02,
                             rot_sigma_deg=0.5, trans_sigma=0.1, seed=5150)
    s = scenegen.make_scene(p)
    cen = oracle.points_to_centred(s.point_offsets(), s.points())
    return s, cen


def _split(s, cen, hidden):
    """Shard A: the voxels none of whose observations is of a scan in
    `hidden`; shard B: the others.  Their CSR slices, every scan kept."""
    vo = s.voxel_off
    bad = np.isin(s.obs_scan, hidden)
    in_a = np.array([not bad[vo[i]:vo[i + 1]].any() for i in range(s.n_voxels)])
    out = []
    for sel in (np.flatnonzero(in_a), np.flatnonzero(~in_a)):
        cnt = np.diff(vo)[sel]
        off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
        idx = np.concatenate([np.arange(vo[i], vo[i + 1]) for i in sel])
        out.append((off, s.obs_scan[idx], cen[idx]))
    return out


# mu follows the gain ratio, a quotient of a small cost difference: its
# rounding is the costs' relative rounding times c / (c - c')
@pytest.mark.parametrize("precision,rot_tol,tr_tol,cost_tol,mu_tol", [("fp64", 1e-10, 1e-9, 1e-11, 1e-6),
                                                                      ("mixed", 1e-6, 1e-5, 1e-6, 1e-2)])
def test_two_shards_follow_the_unsharded_solve(mm, precision, rot_tol, tr_tol, cost_tol, mu_tol):
    prec = mm.BA_MIXED if precision == "mixed" else mm.BA_FP64
    s, cen = _scene()
    # shard A observes neither scan 3 nor scan 4: only the totals say they move
    hidden = [3, 4]
    parts = _split(s, cen, hidden)
    assert 0.2 < len(parts[0][0]) / s.n_voxels < 0.9
    with mm.BundleAdjuster(precision=prec) as U, mm.BundleAdjuster(precision=prec) as A, \
            mm.BundleAdjuster(precision=prec) as B:
        U.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        for h, (vo, os_, ag) in zip((A, B), parts):
            h.load_observations(s.n_scans, vo, os_, ag, s.pose_init)
        ga, ca = A.shard_partials()
        gb, cb = B.shard_partials()
        assert not ga[hidden].any() and gb[hidden].any()
        assert ca + cb == pytest.approx(U.cost(), rel=cost_tol)
        for h in (A, B):
            h.shard_set_totals(ga + gb, ca + cb)
        accepted = 0
        for k in range(8):
            ta, tb = A.shard_trial(), B.shard_trial()
            acc_a, acc_b = A.shard_decide(ta + tb), B.shard_decide(ta + tb)
            st = U.iterate(1)
            assert acc_a == acc_b == bool(st["last_accepted"]), k
            PA, PB = A.poses(), B.poses()
            np.testing.assert_array_equal(PA, PB)
            r, t = pose_errors(PA, U.poses())
            assert r < rot_tol and t < tr_tol, (k, r, t)
            if acc_a:
                accepted += 1
                ga, _ = A.shard_partials()
                gb, _ = B.shard_partials()
                for h in (A, B):
                    h.shard_set_totals(ga + gb, ta + tb)
                assert ta + tb == pytest.approx(st["cost"], rel=cost_tol)
            sa, sb = A.stats(), B.stats()
            assert sa["mu"] == sb["mu"] and sa["mu"] == pytest.approx(st["mu"], rel=mu_tol)
        assert accepted >= 6
