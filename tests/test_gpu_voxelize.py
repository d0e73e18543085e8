"""Preprocessing on the GPU (ba_voxelize: L1 voxelisation, bottom-up levels,
selection; Sec. IV-B, Eq. 4-5, Algorithm 1) against the CPU oracle: the
integer structure (voxels, levels, indices, which scan observes what) bit
for bit, clusters to FP64 rounding (the recursive-summation bound), selection decisions except eigenvalue
near-ties; and the voxelised scans loaded straight into a solve."""
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


def _scan_points(s):
    npo = s.params.pts_per_obs
    order = np.argsort(s.obs_scan, kind="stable")
    P = s.points().reshape(s.n_obs, npo, 3)[order].reshape(-1, 3)
    counts = np.bincount(s.obs_scan, minlength=s.n_scans) * npo
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64), P


@pytest.fixture(scope="module")
def scans():
    s = scenegen.make_scene(scenegen.config("tiny"))
    spo, P = _scan_points(s)
    return s, spo, P


def _same_structure(a, b):
    for k in ("voxel_off", "obs_scan", "level", "index"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


EPS = np.finfo(np.float64).eps


def _close_clusters(got, ref, d):
    """Clusters agree to FP64 rounding.  Both sides sum the same N terms in
    different orders (the GPU as deviations from a run's first point over
    fixed chunks, the oracle as mean then scatter about it); every deviation
    is shorter than the voxel diagonal sqrt(3) d_k, so each side's scatter
    entry is within the recursive-summation bound N eps * N 3 d_k^2 of the
    exact value, and each mean within N eps (|m| + sqrt(3) d_k)."""
    n = ref["agg"][:, 9]
    np.testing.assert_array_equal(got["agg"][:, 9], n)
    dk = d * 2.0 ** (np.repeat(ref["level"], np.diff(ref["voxel_off"])) - 1)
    tol_s = 2 * (n + 1) * EPS * 3 * n * dk**2
    err_s = np.abs(got["agg"][:, :6] - ref["agg"][:, :6])
    assert np.all(err_s <= tol_s[:, None]), np.max(err_s / tol_s[:, None])
    m = ref["agg"][:, 6:9]
    tol_m = 2 * n * EPS * (np.abs(m).max(axis=1) + np.sqrt(3) * dk)
    err_m = np.abs(got["agg"][:, 6:9] - m)
    assert np.all(err_m <= tol_m[:, None]), np.max(err_m / tol_m[:, None])


@pytest.mark.parametrize("d,levels", [(1.0, 3), (0.37, 2), (2.5, 1)])
def test_voxelize_matches_oracle(mm, scans, d, levels):
    s, spo, P = scans
    got = mm.voxelize(spo, P, s.pose_gt, d, levels=levels)
    ref = oracle.voxelize(spo, P, s.pose_gt, d, levels=levels)
    _same_structure(got, ref)
    _close_clusters(got, ref, d)
    assert got["launches"] > 0


def test_selection_matches_oracle_up_to_ties(mm, scans):
    s, spo, P = scans
    d, levels, tau = 1.0, 3, 0.05
    got = mm.voxelize(spo, P, s.pose_init, d, levels=levels, tau=tau, min_obs=2)
    ref = oracle.voxelize(spo, P, s.pose_init, d, levels=levels, tau=tau, min_obs=2)
    allv = oracle.voxelize(spo, P, s.pose_init, d, levels=levels, min_obs=2)
    key = lambda v: {(int(l), tuple(int(x) for x in i)) for l, i in zip(v["level"], v["index"])}
    diff = key(got) ^ key(ref)
    # a differing decision must be a near-tie of lambda0 against tau lambda1
    where = {(int(l), tuple(int(x) for x in i)): n for n, (l, i) in enumerate(zip(allv["level"], allv["index"]))}
    for k in diff:
        n = where[k]
        o0, o1 = allv["voxel_off"][n], allv["voxel_off"][n + 1]
        pts = []
        for o in range(o0, o1):
            T = s.pose_init[allv["obs_scan"][o]]
            c = allv["agg"][o]
            R, t = T[:9].reshape(3, 3), T[9:]
            S = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
            pts.append((R @ S @ R.T, R @ c[6:9] + t, c[9]))
        n_tot = sum(p[2] for p in pts)
        cen = sum(p[2] * p[1] for p in pts) / n_tot
        A = sum(p[0] + p[2] * np.outer(p[1] - cen, p[1] - cen) for p in pts) / n_tot
        lam = np.linalg.eigvalsh(A)
        assert abs(lam[0] - tau * lam[1]) <= 1e-9 * lam[2], (k, lam)
    # every difference was checked to be a tie above; they are rare
    assert len(diff) <= max(2, len(allv["level"]) // 100)
    assert 0 < len(got["level"]) < len(allv["level"])


def test_device_inputs_equal_host_inputs(mm, scans):
    import torch
    s, spo, P = scans
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    a = mm.voxelize(spo, P, s.pose_gt, 1.0, levels=2)
    b = mm.voxelize(dev(spo), dev(P), dev(s.pose_gt), 1.0, levels=2, out="device")
    _same_structure(a, {k: v.cpu().numpy() for k, v in b.items() if hasattr(v, "cpu")})
    np.testing.assert_array_equal(a["agg"], b["agg"].cpu().numpy())


def test_voxelize_edge_cases_and_errors(mm, scans):
    s, spo, P = scans
    # scans without points
    spo2 = spo.copy()
    spo2[3] = spo2[2]  # scan 2 gets no points... scan 3 starts where scan 2 did
    spo2 = np.maximum.accumulate(spo2)
    got = mm.voxelize(spo2, P, s.pose_gt, 1.0, levels=2)
    ref = oracle.voxelize(spo2, P, s.pose_gt, 1.0, levels=2)
    _same_structure(got, ref)
    # no points at all
    empty = mm.voxelize(np.zeros(s.n_scans + 1, np.int64), np.zeros((0, 3)), s.pose_gt, 1.0, levels=3)
    assert len(empty["level"]) == 0 and list(empty["voxel_off"]) == [0]
    # malformed offsets, out-of-range index, bad settings
    bad = spo.copy()
    bad[4] = bad[3] - 1
    with pytest.raises(mm.BAError) as e:
        mm.voxelize(bad, P, s.pose_gt, 1.0)
    assert e.value.status == 1
    far = P.copy()
    far[7] = [5.0e6, 0.0, 0.0]
    with pytest.raises(mm.BAError) as e:
        mm.voxelize(spo, far, s.pose_gt, 1.0)
    assert e.value.status == 7 and "point 7" in str(e.value)
    with pytest.raises(mm.BAError):
        mm.voxelize(spo, P, s.pose_gt, -1.0)
    with pytest.raises(mm.BAError):
        mm.voxelize(spo, P, s.pose_gt, 1.0, levels=0)


@pytest.mark.parametrize("batch", ["whole_scans", "split_scans"])
def test_loader_batches_match_oracle(mm, scans, batch):
    """The adaptive loader (Sec. IV-B): host points in batches (whole scans,
    or batches shorter than a scan so that scans are split and their pieces
    merged) give the oracle's structure and clusters."""
    s, spo, P = scans
    per_scan = int(np.diff(spo).max())
    bp = 3 * per_scan + 17 if batch == "whole_scans" else max(1, per_scan // 3)
    got = mm.voxelize(spo, P, s.pose_gt, 1.0, levels=3, batch_points=bp)
    ref = oracle.voxelize(spo, P, s.pose_gt, 1.0, levels=3)
    assert got["batches"] >= (len(P) + bp - 1) // bp > 1
    _same_structure(got, ref)
    _close_clusters(got, ref, 1.0)


def test_loader_device_batches_and_pinned_host(mm, scans):
    """Device points processed in batches, and pinned host points, equal the
    single pass in structure; a bad point in a later batch is reported by its
    global index."""
    import torch
    s, spo, P = scans
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    one = mm.voxelize(dev(spo), dev(P), dev(s.pose_gt), 0.5, levels=2, out="device")
    assert one["batches"] == 1
    many = mm.voxelize(dev(spo), dev(P), dev(s.pose_gt), 0.5, levels=2, out="device", batch_points=len(P) // 7)
    assert many["batches"] >= 7
    _same_structure({k: v.cpu().numpy() for k, v in one.items() if hasattr(v, "cpu")},
                    {k: v.cpu().numpy() for k, v in many.items() if hasattr(v, "cpu")})
    pinned = torch.from_numpy(P).pin_memory()
    h = mm.voxelize(spo, pinned.numpy(), s.pose_gt, 0.5, levels=2, batch_points=len(P) // 5)
    _same_structure(h, {k: v.cpu().numpy() for k, v in one.items() if hasattr(v, "cpu")})
    far = P.copy()
    q = len(P) - 3
    far[q] = [5.0e6, 0.0, 0.0]
    with pytest.raises(mm.BAError) as e:
        mm.voxelize(spo, far, s.pose_gt, 1.0, batch_points=len(P) // 4)
    assert e.value.status == 7 and f"point {q}" in str(e.value)
    with pytest.raises(mm.BAError):
        mm.voxelize(spo, P, s.pose_gt, 1.0, alpha=0.0)


def _near(poses, rot_rad, trans_m, seed):
    """poses with a small rotation (Exp of a random axis) and translation error"""
    rng = np.random.default_rng(seed)
    out = poses.copy()
    for j in range(1, len(poses)):
        phi = rng.normal(size=3) * rot_rad
        out[j, :9] = (oracle.exp_so3(phi) @ poses[j, :9].reshape(3, 3)).ravel()
        out[j, 9:] += rng.normal(size=3) * trans_m
    return out


def test_voxelised_scans_solve(mm, scans):
    """Raw scans -> voxels (on the device, with selection, grouped at poses
    near the truth) -> loaded from device memory -> solved from the scene's
    perturbed poses: the poses approach the ground truth and the cost at the
    result agrees with the oracle."""
    import torch
    s, spo, P = scans
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    grouping = _near(s.pose_gt, 1e-3, 5e-3, 11)
    v = mm.voxelize(dev(spo), dev(P), dev(grouping), 1.0, levels=2, tau=0.1, min_obs=2, out="device")
    with mm.BundleAdjuster(precision=mm.BA_FP64, max_iters=60) as ba:
        ba.load_observations(s.n_scans, v["voxel_off"], v["obs_scan"], v["agg"], dev(s.pose_init))
        st = ba.solve()
        poses = ba.poses()
        cost = ba.cost()
    r0, t0 = pose_errors(s.pose_init, s.pose_gt)
    r1, t1 = pose_errors(poses, s.pose_gt)
    assert r1 < 0.2 * r0 and t1 < 0.2 * t0, (r0, r1, t0, t1)
    prob = oracle.ObsProblem(s.n_scans, v["voxel_off"].cpu().numpy(), v["obs_scan"].cpu().numpy(),
                             v["agg"].cpu().numpy())
    c_ref, _ = oracle.voxel_pass(prob, poses)
    assert cost == pytest.approx(c_ref, rel=1e-10)
    assert st["accepted"] > 0


def _planar_decisions(voxel_off, obs_scan, agg, poses, tau, min_obs, idx):
    """Keep decision (and whether it is a near-tie) of voxels idx from their
    clusters at the poses, in FP64 numpy: covariance of the voxel's world
    points (Eq. 1-2) and numpy.linalg.eigvalsh."""
    keep, tie = [], []
    for v in idx:
        o0, o1 = voxel_off[v], voxel_off[v + 1]
        if o1 - o0 < min_obs:
            keep.append(False)
            tie.append(False)
            continue
        c = agg[o0:o1]
        T = poses[obs_scan[o0:o1]]
        R, t = T[:, :9].reshape(-1, 3, 3), T[:, 9:]
        S = c[:, [0, 1, 2, 1, 3, 4, 2, 4, 5]].reshape(-1, 3, 3)
        w = np.einsum("kab,kb->ka", R, c[:, 6:9]) + t
        n = c[:, 9]
        m = (n[:, None] * w).sum(0) / n.sum()
        d = w - m
        A = (np.einsum("kab,kbc,kdc->ad", R, S, R) + np.einsum("k,ka,kb->ab", n, d, d)) / n.sum()
        lam = np.linalg.eigvalsh(A)
        keep.append(lam[0] < tau * lam[1])
        tie.append(abs(lam[0] - tau * lam[1]) <= 1e-9 * lam[2])
    return np.array(keep), np.array(tie)


def test_full_size_sampled_parity(mm):
    """The bench's workload and launch configuration (the 1,000-scan scene's
    120M raw points on the device, d = 0.5 m, 3 levels, tau = 0.1, min_obs = 2):
    every observation of three sampled scans equals the oracle run on that
    scan's points alone (clusters of one scan depend on its points only);
    sampled voxels' selection decisions equal the FP64 decision from their
    clusters (up to near-ties); host-batched input gives the same output."""
    import torch
    s = scenegen.make_scene(scenegen.config("mid"))
    npo = s.params.pts_per_obs
    P = torch.empty((s.n_obs * npo, 3), dtype=torch.float64, device="cuda")
    s.points_device(0, s.n_obs, P)
    order = torch.from_numpy(np.argsort(s.obs_scan, kind="stable")).cuda()
    P = P.view(s.n_obs, npo, 3)[order].reshape(-1, 3).contiguous()
    counts = np.bincount(s.obs_scan, minlength=s.n_scans) * npo
    spo = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    dspo, dT = torch.from_numpy(spo).cuda(), torch.from_numpy(s.pose_init).cuda()
    d, levels, tau, min_obs = 0.5, 3, 0.1, 2
    host = lambda r: {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in r.items()}
    allv = host(mm.voxelize(dspo, P, dT, d, levels=levels, out="device"))
    sel = host(mm.voxelize(dspo, P, dT, d, levels=levels, tau=tau, min_obs=min_obs, out="device"))
    rng = np.random.default_rng(7)
    vox_of_obs = np.repeat(np.arange(len(allv["level"])), np.diff(allv["voxel_off"]))
    for j in rng.choice(s.n_scans, 3, replace=False):
        Pj = P[spo[j]:spo[j + 1]].cpu().numpy()
        ref = oracle.voxelize(np.array([0, len(Pj)], np.int64), Pj, s.pose_init[j:j + 1], d, levels=levels)
        mine = np.nonzero(allv["obs_scan"] == j)[0]
        assert len(mine) == len(ref["level"])
        v = vox_of_obs[mine]
        key_got = np.column_stack([allv["level"][v], allv["index"][v]])
        key_ref = np.column_stack([ref["level"], ref["index"]])
        np.testing.assert_array_equal(key_got, key_ref)
        got_one = {"agg": allv["agg"][mine], "level": ref["level"], "voxel_off": np.arange(len(mine) + 1)}
        _close_clusters(got_one, {"agg": ref["agg"], "level": ref["level"], "voxel_off": np.arange(len(mine) + 1)}, d)
    # selection: sampled voxels of the unselected output
    idx = rng.choice(len(allv["level"]), 4000, replace=False)
    keep, tie = _planar_decisions(allv["voxel_off"], allv["obs_scan"], allv["agg"], s.pose_init, tau, min_obs, idx)
    kept = {(int(l), *map(int, i)) for l, i in zip(sel["level"], sel["index"])}
    for v, k, t in zip(idx, keep, tie):
        if t:
            continue
        assert ((int(allv["level"][v]), *map(int, allv["index"][v])) in kept) == k, v
    assert keep.sum() > 50 and (~keep).sum() > 50
    # the loader from pinned host memory, in batches
    Ph = P.cpu().pin_memory()
    hb = mm.voxelize(spo, Ph.numpy(), s.pose_init, d, levels=levels, tau=tau, min_obs=min_obs)
    assert hb["batches"] > 1
    _same_structure(hb, sel)
