"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances for the FP64 path: poses within 1e-9 rad and 1e-8 m, cost within a
relative 1e-10.  Per-voxel and per-scan quantities are compared element by
element; their tolerances follow from the same rounding budget (each is a sum
of a few hundred FP64 terms taken in a different order on each side).
"""
import zlib

import numpy as np
import pytest

import oracle
import scenegen
from tests._util import pose_errors, tiny_scene

pytestmark = pytest.mark.gpu

ROT_TOL, TRANS_TOL, COST_TOL = 1e-9, 1e-8, 1e-10


@pytest.fixture(scope="module")
def mm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2608_14266_gb300 as mm
    assert torch.cuda.is_available()
    return mm


def _solver(mm, s, cen, **cfg):
    ba = mm.BundleAdjuster(**cfg)
    ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
    return ba


def _compare_planes(gpu, ref):
    np.testing.assert_allclose(gpu[:, 0], ref[:, 0], rtol=1e-9, atol=1e-15)
    scale = np.abs(ref[:, 2]).max()
    np.testing.assert_allclose(gpu[:, 1:3], ref[:, 1:3], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(gpu[:, 6:9], ref[:, 6:9], rtol=0, atol=1e-10)
    gap = (ref[:, 1] - ref[:, 0]) / ref[:, 2]
    ok = gap > 1e-6
    dots = np.abs(np.sum(gpu[:, 3:6] * ref[:, 3:6], axis=1))
    assert np.all(dots[ok] > 1 - 1e-10)


def test_point_clusters_match_oracle(mm):
    import torch
    s, pts, po, raw, cen = tiny_scene()
    dev = torch.device("cuda")
    out = torch.empty((s.n_obs, 10), dtype=torch.float64, device=dev)
    mm.ba_aggregate_points(torch.from_numpy(po).to(dev), torch.from_numpy(pts).to(dev), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got[:, 9], cen[:, 9])
    np.testing.assert_allclose(got[:, 6:9], cen[:, 6:9], rtol=0, atol=1e-13)
    scale = np.abs(cen[:, :6]).max(axis=1, keepdims=True)
    assert np.all(np.abs(got[:, :6] - cen[:, :6]) <= 1e-13 * scale)


def test_point_clusters_edge_cases_match_oracle(mm):
    """Clusters the fixed-point sums do not fit, next to ones they do: an
    observation whose only far point sits on the second lane of its pair, a
    first point at the origin, a tiny first point with metre-sized others,
    more than 2^14 points, points near the scan origin with a 3 m spread,
    coordinates crossing zero, millimetre clusters, far clusters (30 km), one
    and two points.  Checked against the oracle within its own FP64 rounding
    (eps times the coordinates' size per term)."""
    import torch
    rng = np.random.default_rng(11)
    obs = []
    base = rng.normal(0, 0.3, (8, 3)) + np.array([40.0, -20.0, 5.0])
    far = base.copy()
    far[3] += np.array([0.0, 900.0, 0.0])  # |d| past the bound, handled by lane 1
    obs += [far, base]
    z = rng.normal(0, 0.5, (12, 3))
    z[0] = 0.0
    obs.append(z)  # first point at the origin
    t = rng.normal(0, 1.0, (10, 3))
    t[0] = np.array([1e-6, -2e-6, 3e-6])
    obs.append(t)  # first point far smaller than the others
    obs.append(rng.normal(0, 0.5, (20000, 3)) + np.array([10.0, 10.0, 2.0]))  # more than 2^14 points
    obs.append(rng.uniform(-3.0, 3.0, (40, 3)))  # near the origin, 3 m spread
    c = rng.normal(0, 0.4, (33, 3))
    c[:, 0] += 0.05
    obs.append(c)  # x crossing zero
    obs.append(rng.normal(0, 1e-4, (25, 3)) + 1e-3)  # millimetre cluster
    obs.append(rng.normal(0, 1.0, (30, 3)) + np.array([3.0e4, -2.5e4, 10.0]))  # 30 km away
    obs.append(np.array([[1.5, -2.5, 0.25]]))
    obs.append(np.array([[1.5, -2.5, 0.25], [1.75, -2.0, 0.5]]))
    for _ in range(40):
        obs.append(rng.normal(0, 0.3, (int(rng.integers(3, 64)), 3)) + rng.uniform(-200, 200, 3))
    po = np.concatenate([[0], np.cumsum([len(o) for o in obs])]).astype(np.int64)
    pts = np.concatenate(obs)
    dev = torch.device("cuda")
    out = torch.empty((len(obs), 10), dtype=torch.float64, device=dev)
    mm.ba_aggregate_points(torch.from_numpy(po).to(dev), torch.from_numpy(pts).to(dev), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle.points_to_centred(po, pts)
    np.testing.assert_array_equal(got[:, 9], ref[:, 9])
    eps = np.finfo(np.float64).eps
    for i, o in enumerate(obs):
        big = np.abs(o).max()
        spread = np.ptp(o, axis=0).max() if len(o) > 1 else 0.0
        n = len(o)
        assert np.abs(got[i, 6:9] - ref[i, 6:9]).max() <= 1e-13 + 4 * n * eps * big, i
        scale = max(np.abs(ref[i, :6]).max(), 1e-300)
        tol = 1e-13 * scale + 8 * n * eps * big * spread
        assert np.abs(got[i, :6] - ref[i, :6]).max() <= tol, (i, got[i], ref[i])


@pytest.mark.parametrize("which", ["init", "gt"])
def test_voxel_pass_matches_oracle(mm, which):
    s, pts, po, raw, cen = tiny_scene()
    poses = s.pose_init if which == "init" else s.pose_gt
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    c_ref, planes_ref = oracle.voxel_pass(prob, poses)
    with mm.BundleAdjuster() as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, poses)
        assert ba.cost() == pytest.approx(c_ref, rel=COST_TOL)
        _compare_planes(ba.planes(), planes_ref)


def test_gradient_and_hessian_match_oracle(mm):
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    for gn in (False, True):
        _, planes = oracle.voxel_pass(prob, s.pose_init)
        g_ref, H_ref = oracle.grad_hess(prob, s.pose_init, planes, gauss_newton=gn)
        with mm.BundleAdjuster(hessian_mode=int(gn)) as ba:
            ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
            g, H = ba.gradient()
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-10 * np.abs(g_ref).max())
        for j in range(s.n_scans):
            np.testing.assert_allclose(H[j], H_ref[j], rtol=0, atol=1e-11 * np.abs(H_ref[j]).max())


def test_points_path_equals_cluster_path(mm):
    s, pts, po, raw, cen = tiny_scene()
    with mm.BundleAdjuster() as a, mm.BundleAdjuster() as b:
        a.load_points(s.n_scans, s.voxel_off, s.obs_scan, po, pts, s.pose_init)
        b.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        assert a.cost() == pytest.approx(b.cost(), rel=1e-13)
        a.iterate(3)
        b.iterate(3)
        r, t = pose_errors(a.poses(), b.poses())
        assert r < 1e-12 and t < 1e-11


def test_raw_sum_input(mm):
    """Raw sums are converted with the documented fma rule; the oracle applies
    the same rule, so both sides see identical centred clusters."""
    s, pts, po, raw, cen = tiny_scene()
    conv = oracle.raw_to_centred(raw)
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, conv)
    c_ref, planes_ref = oracle.voxel_pass(prob, s.pose_init)
    with mm.BundleAdjuster() as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, raw, s.pose_init, agg_form=mm.BA_AGG_RAW_SUMS)
        assert ba.cost() == pytest.approx(c_ref, rel=COST_TOL)
        _compare_planes(ba.planes(), planes_ref)


def test_each_iteration_from_the_oracle_state(mm):
    """Feed the oracle's state (poses, mu, nu) into one GPU iteration, for each
    of the first 12 iterations of the tiny workload."""
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    lm = oracle.LM(prob, s.pose_init)
    with mm.BundleAdjuster() as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        for k in range(12):
            ba.set_state(lm.poses, lm.mu, lm.nu)
            assert ba.cost() == pytest.approx(lm.cost, rel=COST_TOL)
            st = ba.iterate(1)
            acc = lm.step()
            assert bool(st["last_accepted"]) == acc
            assert st["last_trial_cost"] == pytest.approx(lm.st.last_trial_cost, rel=COST_TOL)
            assert st["last_pred"] == pytest.approx(lm.st.last_pred, rel=1e-8)
            assert st["mu"] == pytest.approx(lm.mu, rel=1e-8)
            r, t = pose_errors(ba.poses(), lm.poses)
            assert r < ROT_TOL and t < TRANS_TOL, (k, r, t)


def test_twenty_iterations_match_oracle(mm):
    """The tiny workload end to end: raw points, 20 LM iterations."""
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    lm = oracle.LM(prob, s.pose_init)
    for _ in range(20):
        lm.step()
    with mm.BundleAdjuster() as ba:
        ba.load_points(s.n_scans, s.voxel_off, s.obs_scan, po, pts, s.pose_init)
        st = ba.iterate(20)
        assert st["iters"] == 20 and st["accepted"] == lm.st.accepted
        assert st["cost"] == pytest.approx(lm.cost, rel=COST_TOL)
        r, t = pose_errors(ba.poses(), lm.poses)
        assert r < ROT_TOL and t < TRANS_TOL, (r, t)


def test_solve_stops_like_the_oracle(mm):
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    lm = oracle.LM(prob, s.pose_init, rel_tol=1e-3, max_iters=60)
    lm.solve()
    with mm.BundleAdjuster(rel_tol=1e-3, max_iters=60) as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        st = ba.solve()
        assert st["iters"] == lm.st.iters and st["converged"] == lm.st.converged
        r, t = pose_errors(ba.poses(), lm.poses)
        assert r < ROT_TOL and t < TRANS_TOL
        # iterations after the stop are real iterations again under ba_iterate
        st2 = ba.iterate(2)
        assert st2["iters"] == st["iters"] + 2


def _edge_problem(rng, n_scans, lens, pts_per_obs=12):
    """Random planar clusters with given per-voxel observation counts."""
    import oracle as orc
    voxel_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n_obs = int(voxel_off[-1])
    obs_scan = np.empty(n_obs, np.int32)
    pts = []
    poses = np.zeros((n_scans, 12))
    for j in range(n_scans):
        poses[j, :9] = orc.exp_so3(rng.normal(size=3)).ravel()
        poses[j, 9:] = rng.uniform(0, 20, 3)
    for i, L in enumerate(lens):
        c = rng.uniform(0, 20, 3)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        e1 = np.cross(n, rng.normal(size=3))
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(n, e1)
        scans = rng.choice(n_scans, size=L, replace=L > n_scans)
        for k in range(L):
            o = voxel_off[i] + k
            obs_scan[o] = scans[k]
            ab = rng.uniform(-0.5, 0.5, (pts_per_obs, 2))
            w = c + ab[:, :1] * e1 + ab[:, 1:] * e2 + rng.normal(0, 0.01, (pts_per_obs, 1)) * n
            P = poses[scans[k]]
            pts.append((w - P[9:]) @ P[:9].reshape(3, 3))
    pts = np.concatenate(pts)
    po = np.arange(n_obs + 1, dtype=np.int64) * pts_per_obs
    # perturb the poses
    init = poses.copy()
    for j in range(1, n_scans):
        init[j] = orc.retract(poses[j], np.concatenate([rng.normal(0, 0.005, 3), rng.normal(0, 0.02, 3)]))
    return voxel_off, obs_scan, po, pts, init


@pytest.mark.parametrize("case", ["single_obs_voxels", "long_voxels", "ragged_37", "idle_scans", "one_scan",
                                  "no_fixed_scan", "one_voxel", "two_scans"])
def test_edge_cases_match_oracle(mm, case):
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    cfg = {}
    n_idle = 0
    if case == "single_obs_voxels":
        n_scans, lens = 6, [1] * 40 + list(rng.integers(2, 9, 60))
    elif case == "long_voxels":
        n_scans, lens = 8, [300, 1, 77, 33, 32, 31, 64, 65] + list(rng.integers(3, 12, 50))
    elif case == "ragged_37":
        n_scans, lens = 7, list(rng.integers(2, 15, 37))
    elif case == "idle_scans":  # scans 5..9 observe nothing
        n_scans, lens, n_idle = 5, list(rng.integers(2, 6, 80)), 5
    elif case == "one_scan":
        n_scans, lens = 1, list(rng.integers(1, 4, 30))
        cfg = {"fixed_scan": -1}
    elif case == "one_voxel":  # the whole problem is one plane seen by four scans
        n_scans, lens = 4, [4]
    elif case == "two_scans":
        n_scans, lens = 2, list(rng.integers(1, 3, 25))
    else:
        n_scans, lens = 6, list(rng.integers(3, 10, 70))
        cfg = {"fixed_scan": -1}
    voxel_off, obs_scan, po, pts, init = _edge_problem(rng, n_scans, lens)
    if n_idle:
        idle = np.tile(np.concatenate([np.eye(3).ravel(), np.zeros(3)]), (n_idle, 1))
        init = np.concatenate([init, idle])
        n_scans += n_idle
    cen = oracle.points_to_centred(po, pts)
    prob = oracle.ObsProblem(n_scans, voxel_off, obs_scan, cen)
    lm = oracle.LM(prob, init, fixed_scan=cfg.get("fixed_scan", 0))
    with mm.BundleAdjuster(**cfg) as ba:
        ba.load_points(n_scans, voxel_off, obs_scan, po, pts, init)
        assert ba.cost() == pytest.approx(lm.cost, rel=COST_TOL)
        _compare_planes(ba.planes(), lm.planes)
        for k in range(5):
            c_prev = lm.cost
            st = ba.iterate(1)
            acc = lm.step()
            if bool(st["last_accepted"]) != acc:
                # only a near-tie may be decided differently: the cost change is
                # within the rounding budget (e.g. a single scan, whose pose does
                # not change the cost at all); then continue from the oracle state
                assert abs(lm.st.last_trial_cost - c_prev) <= COST_TOL * c_prev, k
                assert st["last_trial_cost"] == pytest.approx(lm.st.last_trial_cost, rel=COST_TOL)
                ba.set_state(lm.poses, lm.mu, lm.nu)
                continue
            assert st["cost"] == pytest.approx(lm.cost, rel=COST_TOL)
            r, t = pose_errors(ba.poses(), lm.poses)
            assert r < ROT_TOL and t < TRANS_TOL, (k, r, t)
        if case == "idle_scans":
            np.testing.assert_array_equal(ba.poses()[5:], init[5:])


def _degenerate_problem(rng, n_scans=6, n_vox=64):
    """Planar voxels whose clusters are rank-deficient: one point (zero
    scatter), two points (rank one), points on a line, points on a line
    with noise along the plane normal (rank two), and noise-free points on
    the plane laid out so that the scan frame's z axis is the normal (the
    scatter's z row zero up to rounding)."""
    import oracle as orc
    poses = np.zeros((n_scans, 12))
    for j in range(n_scans):
        poses[j, :9] = orc.exp_so3(rng.normal(size=3)).ravel()
        poses[j, 9:] = rng.uniform(0, 20, 3)
    lens = rng.integers(3, 9, n_vox)
    voxel_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    obs_scan = np.empty(int(voxel_off[-1]), np.int32)
    pts, npts = [], []
    for i, L in enumerate(lens):
        scans = rng.choice(n_scans, size=L, replace=L > n_scans)
        R0 = poses[scans[0], :9].reshape(3, 3)
        n = R0[:, 2] if i % 2 else rng.normal(size=3)  # odd voxels: normal along scan z of their first scan
        n /= np.linalg.norm(n)
        e1 = np.cross(n, rng.normal(size=3))
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(n, e1)
        c = rng.uniform(0, 20, 3)
        for k in range(L):
            o = voxel_off[i] + k
            obs_scan[o] = scans[k]
            shape = (i + k) % 5
            if shape == 0:  # one point
                ab = rng.uniform(-0.5, 0.5, (1, 2))
                off = rng.normal(0, 0.01, (1, 1))
            elif shape == 1:  # two points
                ab = rng.uniform(-0.5, 0.5, (2, 2))
                off = rng.normal(0, 0.01, (2, 1))
            elif shape == 2:  # on a line
                t = rng.uniform(-0.5, 0.5, (7, 1))
                ab = t * rng.normal(size=(1, 2))
                off = np.zeros((7, 1))
            elif shape == 3:  # a line, noise along the normal
                t = rng.uniform(-0.5, 0.5, (7, 1))
                ab = t * rng.normal(size=(1, 2))
                off = rng.normal(0, 0.01, (7, 1))
            else:  # on the plane, no noise
                ab = rng.uniform(-0.5, 0.5, (9, 2))
                off = np.zeros((9, 1))
            w = c + ab[:, :1] * e1 + ab[:, 1:] * e2 + off * n
            P = poses[scans[k]]
            pts.append((w - P[9:]) @ P[:9].reshape(3, 3))
            npts.append(len(w))
    pts = np.concatenate(pts)
    po = np.concatenate([[0], np.cumsum(npts)]).astype(np.int64)
    init = poses.copy()
    for j in range(1, n_scans):
        init[j] = orc.retract(poses[j], np.concatenate([rng.normal(0, 0.005, 3), rng.normal(0, 0.02, 3)]))
    return voxel_off, obs_scan, po, pts, init


def test_rank_deficient_clusters_match_oracle(mm):
    """Clusters whose scatter is zero, rank one or rank two: the voxel pass's
    factored scatters (pivoted LDL^T) and its eigen-solve against the oracle,
    then five LM iterations."""
    rng = np.random.default_rng(2024)
    n_scans = 6
    voxel_off, obs_scan, po, pts, init = _degenerate_problem(rng, n_scans)
    cen = oracle.points_to_centred(po, pts)
    lm = oracle.LM(oracle.ObsProblem(n_scans, voxel_off, obs_scan, cen), init)
    with mm.BundleAdjuster() as ba:
        ba.load_points(n_scans, voxel_off, obs_scan, po, pts, init)
        assert ba.cost() == pytest.approx(lm.cost, rel=COST_TOL)
        _compare_planes(ba.planes(), lm.planes)
        for k in range(5):
            st = ba.iterate(1)
            assert bool(st["last_accepted"]) == lm.step(), k
            assert st["cost"] == pytest.approx(lm.cost, rel=COST_TOL)
            r, t = pose_errors(ba.poses(), lm.poses)
            assert r < ROT_TOL and t < TRANS_TOL, (k, r, t)


def _expect_invalid(mm, fn, match):
    with pytest.raises(mm.BAError) as ei:
        fn()
    assert ei.value.status == 1, ei.value
    assert match in str(ei.value), str(ei.value)


def test_invalid_inputs_are_rejected(mm):
    s, pts, po, raw, cen = tiny_scene()
    with mm.BundleAdjuster() as ba:
        with pytest.raises(mm.BAError) as ei:
            ba.iterate(1)
        assert ei.value.status == 4  # nothing loaded
        args = dict(n_scans=s.n_scans, voxel_offsets=s.voxel_off, obs_scan=s.obs_scan, agg=cen, poses=s.pose_init)

        def load(**kw):
            a = dict(args)
            a.update(kw)
            return ba.load_observations(a["n_scans"], a["voxel_offsets"], a["obs_scan"], a["agg"], a["poses"])

        bad = s.voxel_off.copy()
        bad[5] = bad[4]
        _expect_invalid(mm, lambda: load(voxel_offsets=bad), "voxel 4 has no observation")
        bad = s.voxel_off.copy()
        bad[7] = bad[8] + 1
        _expect_invalid(mm, lambda: load(voxel_offsets=bad), "voxel_offsets")
        bad = s.obs_scan.copy()
        bad[11] = s.n_scans
        _expect_invalid(mm, lambda: load(obs_scan=bad), "obs_scan[11]")
        bad = cen.copy()
        bad[13, 9] = 0.0
        _expect_invalid(mm, lambda: load(agg=bad), "cluster 13")
        bad = cen.copy()
        bad[17, 2] = np.nan
        _expect_invalid(mm, lambda: load(agg=bad), "cluster 17")
        bad = s.pose_init.copy()
        bad[3, 0] *= 1.01
        _expect_invalid(mm, lambda: load(poses=bad), "pose 3")
        bad = s.pose_init.copy()
        bad[2, :9] = -bad[2, :9]  # reflection
        _expect_invalid(mm, lambda: load(poses=bad), "pose 2")
        # a failed load leaves nothing loaded; a good load afterwards works
        with pytest.raises(mm.BAError):
            ba.cost()
        load()
        assert ba.cost() > 0


def test_checkpoint_resume_equals_uninterrupted(mm):
    s, pts, po, raw, cen = tiny_scene()
    with mm.BundleAdjuster() as a, mm.BundleAdjuster() as b:
        a.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        b.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        a.iterate(10)
        b.iterate(4)
        saved, st = b.poses(), b.stats()
        b.close()
        # the resumed handle loads the same problem (clusters and initial
        # poses, which fix the layout and so the order of every sum) and
        # takes the saved state
        c = mm.BundleAdjuster()
        c.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        c.set_state(saved, st["mu"], st["nu"])
        c.iterate(6)
        r, t = pose_errors(a.poses(), c.poses())
        assert r < 1e-13 and t < 1e-12
        assert c.cost() == a.cost()
        c.close()


def test_device_inputs_and_outputs(mm):
    import torch
    s, pts, po, raw, cen = tiny_scene()
    dev = torch.device("cuda")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    with mm.BundleAdjuster() as a, mm.BundleAdjuster() as b:
        a.load_observations(s.n_scans, T(s.voxel_off), T(s.obs_scan), T(cen), T(s.pose_init))
        b.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        a.iterate(4)
        b.iterate(4)
        out = torch.empty((s.n_scans, 12), dtype=torch.float64, device=dev)
        a.poses(out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), b.poses())


def _mid_problem():
    p = scenegen.config("mid")
    s = scenegen.make_scene(p)
    pts = s.points()
    po = s.point_offsets()
    return s, pts, po


def test_mid_workload_full_parity(mm):
    """1,000 scans / 50,000 voxels / ~1.2M clusters from ~120M points: every
    plane, every per-scan g and H, and one iteration, element by element."""
    s, pts, po = _mid_problem()
    cen = oracle.points_to_centred(po, pts)
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    lm = oracle.LM(prob, s.pose_init)
    with mm.BundleAdjuster() as ba:
        ba.load_points(s.n_scans, s.voxel_off, s.obs_scan, po, pts, s.pose_init)
        del pts
        assert ba.cost() == pytest.approx(lm.cost, rel=COST_TOL)
        _compare_planes(ba.planes(), lm.planes)
        g, H = ba.gradient()
        np.testing.assert_allclose(g, lm.g, rtol=0, atol=1e-10 * np.abs(lm.g).max())
        Hs = np.abs(lm.H).max(axis=(1, 2), keepdims=True)
        assert np.all(np.abs(H - lm.H) <= 1e-11 * Hs)
        st = ba.iterate(1)
        acc = lm.step()
        assert bool(st["last_accepted"]) == acc
        assert st["cost"] == pytest.approx(lm.cost, rel=COST_TOL)
        r, t = pose_errors(ba.poses(), lm.poses)
        assert r < ROT_TOL and t < TRANS_TOL, (r, t)


def test_allocator_callbacks_and_injected_oom(mm):
    """Device memory through caller callbacks (here PyTorch's caching
    allocator): every allocation is freed through the callback, and an
    allocation that fails (the Nth call returns NULL) makes the load return
    BA_ERR_OOM with nothing leaked; the handle then loads with a working
    allocator."""
    import torch
    s, pts, po, raw, cen = tiny_scene()
    live = {}

    def make(fail_at=None):
        calls = [0]

        def alloc(n, stream):
            calls[0] += 1
            if fail_at is not None and calls[0] == fail_at:
                return 0
            p = torch.cuda.caching_allocator_alloc(n, stream=torch.cuda.current_stream().cuda_stream)
            live[p] = n
            return p

        def free(p, n, stream):
            assert live.pop(p) == n
            torch.cuda.caching_allocator_delete(p)
        return alloc, free, calls

    alloc, free, calls = make()
    with mm.BundleAdjuster(alloc=alloc, free=free) as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        st = ba.iterate(3)
        assert np.isfinite(st["cost"])
        n_allocs = calls[0]
    assert n_allocs > 5 and not live
    for fail_at in (1, n_allocs // 2, n_allocs):
        alloc, free, calls = make(fail_at)
        ba = mm.BundleAdjuster(alloc=alloc, free=free)
        with pytest.raises(mm.BAError) as e:
            ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        assert e.value.status == 2, str(e.value)  # BA_ERR_OOM
        ba.close()
        torch.cuda.synchronize()
        assert not live, fail_at
    # the library's own pool is unaffected, and its cache can be released
    with mm.BundleAdjuster() as ba:
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen, s.pose_init)
        ba.iterate(1)
    from paper_2608_14266_gb300 import _lib
    assert _lib.lib().ba_release_cached_memory(0) == 0
