"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with a retyped copy of itself: each check
uses a closed form, an invariance, a library routine (LAPACK, scipy expm,
numpy.linalg.solve), finite differences or brute force over raw points.
"""
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from tests._util import pose_errors, random_poses_near, skew, tiny_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "planar_grid.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows.append((f[0], *map(float, f[1:])))
    return rows


def _rigid(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    return R, rng.uniform(-30, 30, 3)


def _pose(R, t):
    return np.concatenate([R.reshape(-1), t])


# ---- Eq. 1 / Eq. 2: closed forms -------------------------------------------

@pytest.mark.parametrize("row", [r for r in _golden_rows() if r[0] == "grid"])
def test_grid_closed_form_any_pose(row):
    """Eq. 1 on the planar grid equals delta^2 for any scan pose (golden fixture)."""
    _, delta, l0, l1, l2, _ = row
    rng = np.random.default_rng(7)
    a, b, e = np.meshgrid([-1.0, 0.0, 1.0], [-1.0, 0.0, 1.0], [-delta, delta], indexing="ij")
    plane_pts = np.stack([a.ravel(), b.ravel(), e.ravel()], 1)
    # world frame = some rigid placement of the plane frame; scan pose arbitrary
    Rw, tw = _rigid(rng)
    world = plane_pts @ Rw.T + tw
    Rs, ts = _rigid(rng)
    scan_pts = (world - ts) @ Rs  # p = Rs^T (w - ts)
    po = np.array([0, len(scan_pts)])
    poses = _pose(Rs, ts)[None]
    voxel_off = np.array([0, 1])
    obs_scan = np.array([0], np.int32)
    c_pts, _ = oracle.cost_points(voxel_off, obs_scan, po, scan_pts, poses)
    cen = oracle.points_to_centred(po, scan_pts)
    c_agg, planes = oracle.voxel_pass(oracle.ObsProblem(1, voxel_off, obs_scan, cen), poses)
    assert c_pts == pytest.approx(l0, rel=1e-10, abs=1e-15)
    assert c_agg == pytest.approx(l0, rel=1e-10, abs=1e-15)
    np.testing.assert_allclose(planes[0, :3], [l0, l1, l2], rtol=1e-10)
    # eigenvector of lambda_min is the plane normal (third axis of the plane frame)
    assert abs(planes[0, 3:6] @ Rw[:, 2]) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("row", [r for r in _golden_rows() if r[0] == "two_scan"])
def test_two_scan_closed_form_and_gradient(row):
    """Two scans offset by delta along the normal: lambda_min = delta^2/4 and the
    surrogate gradient of scan B is delta/2 along the normal (golden fixture)."""
    _, delta, l0, _, _, dl = row
    a, b = np.meshgrid([-1.0, 0.0, 1.0], [-1.0, 0.0, 1.0], indexing="ij")
    base = np.stack([a.ravel(), b.ravel(), np.zeros(9)], 1)
    rng = np.random.default_rng(3)
    Rw, tw = _rigid(rng)
    u = Rw[:, 2]
    wA = base @ Rw.T + tw
    wB = wA + delta * u
    RA, tA = _rigid(rng)
    RB, tB = _rigid(rng)
    pA = (wA - tA) @ RA
    pB = (wB - tB) @ RB
    pts = np.concatenate([pA, pB])
    po = np.array([0, 9, 18])
    poses = np.stack([_pose(RA, tA), _pose(RB, tB)])
    voxel_off = np.array([0, 2])
    obs_scan = np.array([0, 1], np.int32)
    cen = oracle.points_to_centred(po, pts)
    prob = oracle.ObsProblem(2, voxel_off, obs_scan, cen)
    c, planes = oracle.voxel_pass(prob, poses)
    assert c == pytest.approx(l0, rel=1e-10)
    g, _ = oracle.grad_hess(prob, poses, planes)
    sign = np.sign(planes[0, 3:6] @ u)
    np.testing.assert_allclose(g[1, 3:], dl * u, atol=1e-12)
    np.testing.assert_allclose(g[0, 3:], -dl * u, atol=1e-12)
    assert sign != 0


def test_points_cost_equals_cluster_cost():
    """Brute-force cost over raw world points = cost from point clusters (Eq. 1-2)."""
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    for poses in (s.pose_gt, s.pose_init):
        c_pts, lam_pts = oracle.cost_points(s.voxel_off, s.obs_scan, po, pts, poses)
        c_agg, planes = oracle.voxel_pass(prob, poses)
        assert c_agg == pytest.approx(c_pts, rel=1e-12)
        np.testing.assert_allclose(planes[:, 0], lam_pts, rtol=1e-9, atol=1e-15)
        # Eq. 1 exactly as printed (raw sums, P/N - v v^T/N^2) loses digits to
        # cancellation (|v/N|^2 ~ 1e3 m^2 against lambda ~ 1e-4 m^2), so its bound
        # is looser: 1e-16 * 1e3 / 1e-4 ~ 1e-9 per voxel.
        c_eq1, _ = oracle.cost_eq1(s.voxel_off, s.obs_scan, raw, poses)
        assert c_eq1 == pytest.approx(c_pts, rel=1e-8)


def test_raw_and_centred_clusters_agree():
    s, pts, po, raw, cen = tiny_scene()
    conv = oracle.raw_to_centred(raw)
    # identical count and mean; scatter equal up to the cancellation of sum pp^T
    np.testing.assert_array_equal(conv[:, 9], cen[:, 9])
    np.testing.assert_allclose(conv[:, 6:9], cen[:, 6:9], rtol=1e-13, atol=1e-12)
    scale = np.abs(raw[:, :6]).max(axis=1, keepdims=True)
    assert np.all(np.abs(conv[:, :6] - cen[:, :6]) <= 1e-13 * scale)
    # the clusters also reproduce plain numpy sums of the raw points
    o = 17
    p = pts[po[o]:po[o + 1]]
    np.testing.assert_allclose(raw[o, 6:9], p.sum(0), rtol=1e-14)
    np.testing.assert_allclose(raw[o, :3], (p[:, :1] * p).sum(0), rtol=1e-13)
    np.testing.assert_allclose(cen[o, :6][[0, 3, 5]], ((p - p.mean(0)) ** 2).sum(0), rtol=1e-12)


# ---- 3x3 eigen-solve ------------------------------------------------------------

def _pack(A):
    return np.array([A[0, 0], A[0, 1], A[0, 2], A[1, 1], A[1, 2], A[2, 2]])


def test_eig3_matches_lapack_on_voxel_covariances():
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    _, planes = oracle.voxel_pass(prob, s.pose_init)
    rng = np.random.default_rng(0)
    mats = []
    for i in range(0, s.n_voxels):
        lo, hi = s.voxel_off[i], s.voxel_off[i + 1]
        world = []
        for o in range(lo, hi):
            P = s.pose_init[s.obs_scan[o]]
            world.append(pts[po[o]:po[o + 1]] @ P[:9].reshape(3, 3).T + P[9:])
        w = np.concatenate(world)
        mats.append(np.cov(w.T, bias=True))
    mats += [rng.normal(size=(3, 3)) for _ in range(50)]
    for k, M in enumerate(mats):
        M = 0.5 * (M + M.T)
        lam, V, _ = oracle.eig3(_pack(M))
        ref, Vr = np.linalg.eigh(M)
        scale = np.abs(ref).max()
        np.testing.assert_allclose(lam, ref, rtol=0, atol=1e-14 * scale)
        np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-14)
        np.testing.assert_allclose(M @ V, V * lam, atol=1e-13 * scale)
        gaps = np.diff(ref)
        for c in range(3):
            gap = min(gaps[c - 1] if c > 0 else np.inf, gaps[c] if c < 2 else np.inf)
            if gap > 1e-6 * scale:
                assert abs(V[:, c] @ Vr[:, c]) == pytest.approx(1.0, abs=1e-10)
        if k < s.n_voxels:
            assert planes[k, 0] == pytest.approx(ref[0], rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("spec", [(3.0, 2.0, 1.0), (1e-6, 1.0, 1.0), (5.0, 5.0, 5.0), (0.0, 0.0, 0.0),
                                  (-2.0, 1e-3, 7.0), (1e-4, 2e-4, 0.1)])
def test_eig3_known_spectrum(spec):
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    for M in (np.diag(spec), Q @ np.diag(spec) @ Q.T):
        lam, V, sweeps = oracle.eig3(_pack(M))
        np.testing.assert_allclose(lam, np.sort(spec), atol=1e-14 * max(1.0, max(abs(x) for x in spec)))
        assert sweeps < 20


# ---- Eq. 3: the MM surrogate ---------------------------------------------------

def test_surrogate_eq3_is_fixed_plane_form():
    """Eq. 3 as printed equals (1/N_i) sum (u^T q - d)^2 with d = u^T c^(l)."""
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    _, planes_l = oracle.voxel_pass(prob, s.pose_init)
    rng = np.random.default_rng(5)
    for k in range(5):
        T = random_poses_near(s.pose_init, rng, 0.01, 0.05)
        a = oracle.surrogate_eq3(s.voxel_off, s.obs_scan, raw, T, planes_l, s.pose_init)
        b = oracle.surrogate_points(s.voxel_off, s.obs_scan, po, pts, T, planes_l)
        assert a == pytest.approx(b, rel=1e-8)


def test_surrogate_touches_and_majorizes():
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    for Tl in (s.pose_init, s.pose_gt):
        c_l, planes_l = oracle.voxel_pass(prob, Tl)
        touch = oracle.surrogate_points(s.voxel_off, s.obs_scan, po, pts, Tl, planes_l)
        assert touch == pytest.approx(c_l, rel=1e-12)
        rng = np.random.default_rng(1)
        for k in range(200):
            sig = 10.0 ** rng.uniform(-6, -1)
            T = random_poses_near(Tl, rng, sig, sig)
            cm = oracle.surrogate_points(s.voxel_off, s.obs_scan, po, pts, T, planes_l)
            c, _ = oracle.voxel_pass(prob, T)
            assert cm >= c - 1e-12 * c


# ---- derivatives ---------------------------------------------------------------

def _perturb(poses, j, k, h):
    d = np.zeros(6)
    d[k] = h
    out = poses.copy()
    out[j] = oracle.retract(poses[j], d)
    return out


def test_gradient_matches_finite_differences_of_surrogate():
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    Tl = s.pose_init
    _, planes_l = oracle.voxel_pass(prob, Tl)
    g, _ = oracle.grad_hess(prob, Tl, planes_l)
    h = 1e-6
    fd = np.zeros_like(g)
    for j in range(s.n_scans):
        for k in range(6):
            fp = oracle.surrogate_points(s.voxel_off, s.obs_scan, po, pts, _perturb(Tl, j, k, h), planes_l)
            fm = oracle.surrogate_points(s.voxel_off, s.obs_scan, po, pts, _perturb(Tl, j, k, -h), planes_l)
            fd[j, k] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-6 * np.abs(g).max())


def test_gradient_is_tangent_to_true_cost():
    """At T^(l) the surrogate touches the cost, so its gradient is the cost's
    gradient; this also pins the retraction convention (left perturbation)."""
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    Tl = s.pose_init
    _, planes_l = oracle.voxel_pass(prob, Tl)
    g, _ = oracle.grad_hess(prob, Tl, planes_l)
    h = 1e-6
    fd = np.zeros_like(g)
    for j in range(s.n_scans):
        for k in range(6):
            fp, _ = oracle.voxel_pass(prob, _perturb(Tl, j, k, h))
            fm, _ = oracle.voxel_pass(prob, _perturb(Tl, j, k, -h))
            fd[j, k] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-6 * np.abs(g).max())


def _fd_hessian(prob, Tl, planes_l, scans, h=1e-5):
    out = {}
    for j in scans:
        Hfd = np.zeros((6, 6))
        for k in range(6):
            gp, _ = oracle.grad_hess(prob, _perturb(Tl, j, k, h), planes_l)
            gm, _ = oracle.grad_hess(prob, _perturb(Tl, j, k, -h), planes_l)
            Hfd[:, k] = (gp[j] - gm[j]) / (2 * h)
        out[j] = Hfd
    return out


def test_hessian_matches_finite_differences_of_gradient():
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    Tl = s.pose_init
    _, planes_l = oracle.voxel_pass(prob, Tl)
    # The gradient is taken at T near T^(l) with planes frozen at T^(l): this is the
    # surrogate's own gradient field.  Because Exp(a)Exp(b) = Exp(a + b + [a, b]/2 + ...),
    # its FD Jacobian along left perturbations is H plus an antisymmetric term
    # (e_i x e_k) . g_rot / 2, so the symmetric part of the FD Jacobian is H.
    _, H = oracle.grad_hess(prob, Tl, planes_l)
    g, _ = oracle.grad_hess(prob, Tl, planes_l)
    fds = _fd_hessian(prob, Tl, planes_l, range(1, s.n_scans))
    for j, Hfd in fds.items():
        Hs = 0.5 * (Hfd + Hfd.T)
        scale = np.abs(H[j]).max()
        np.testing.assert_allclose(H[j], Hs, rtol=0, atol=2e-6 * scale)


def test_gauss_newton_drops_a_term_the_pins_detect():
    """Dropping the second-order rotation term (Gauss-Newton) fails the FD pin at
    a non-stationary point: the Hessian pin is sensitive to a dropped term."""
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    Tl = s.pose_init
    _, planes_l = oracle.voxel_pass(prob, Tl)
    _, Hgn = oracle.grad_hess(prob, Tl, planes_l, gauss_newton=True)
    fds = _fd_hessian(prob, Tl, planes_l, [1, 2, 3])
    worst = max(np.abs(Hgn[j] - 0.5 * (F + F.T)).max() / np.abs(Hgn[j]).max() for j, F in fds.items())
    assert worst > 1e-4


def test_single_observation_voxel_has_zero_gradient():
    """A voxel seen by one scan contributes no gradient at T^(l)."""
    s, pts, po, raw, cen = tiny_scene()
    o0, o1 = s.voxel_off[0], s.voxel_off[1]
    # keep only the first observation of voxel 0
    voxel_off = np.array([0, 1])
    obs_scan = s.obs_scan[o0:o0 + 1]
    prob = oracle.ObsProblem(s.n_scans, voxel_off, obs_scan, cen[o0:o0 + 1])
    _, planes = oracle.voxel_pass(prob, s.pose_init)
    g, H = oracle.grad_hess(prob, s.pose_init, planes)
    assert np.abs(g).max() < 1e-10 * np.abs(H).max()
    assert np.abs(H[obs_scan[0]]).max() > 0


# ---- solve and retraction -----------------------------------------------------

def test_ldlt6_matches_numpy_solve():
    rng = np.random.default_rng(2)
    for k in range(100):
        B = rng.normal(size=(6, 6)) * 10.0 ** rng.uniform(-3, 3, size=6)
        A = B @ B.T + 1e-3 * np.eye(6)
        b = rng.normal(size=6)
        rc, x = oracle.ldlt6(A, b)
        assert rc == 0
        ref = np.linalg.solve(A, b)
        # forward error bounded by the condition number (both solvers are backward stable)
        bound = 1e-13 * np.linalg.cond(A) * np.linalg.norm(ref)
        assert np.linalg.norm(x - ref) <= bound
    # indefinite and singular matrices are refused
    A = np.eye(6)
    A[3, 3] = -1.0
    assert oracle.ldlt6(A, np.ones(6))[0] == -1
    A[3, 3] = 0.0
    assert oracle.ldlt6(A, np.ones(6))[0] == -1


@pytest.mark.parametrize("mag", [0.0, 1e-12, 1e-8, 9.9e-7, 1.01e-6, 1e-3, 0.3, 2.0, np.pi - 1e-6])
def test_exp_so3(mag):
    rng = np.random.default_rng(4)
    for k in range(5):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        phi = mag * axis
        R = oracle.exp_so3(phi)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-15)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-15)
        np.testing.assert_allclose(R @ oracle.exp_so3(-phi), np.eye(3), atol=1e-15)
        np.testing.assert_allclose(R, scipy.linalg.expm(skew(phi)), atol=2e-15)


def test_retraction_is_left_multiplicative():
    rng = np.random.default_rng(9)
    pose = np.concatenate([oracle.exp_so3(rng.normal(size=3)).ravel(), rng.normal(size=3)])
    d = rng.normal(scale=0.1, size=6)
    out = oracle.retract(pose, d)
    np.testing.assert_allclose(out[:9].reshape(3, 3),
                               scipy.linalg.expm(skew(d[:3])) @ pose[:9].reshape(3, 3), atol=1e-14)
    np.testing.assert_allclose(out[9:], pose[9:] + d[3:], atol=1e-15)


# ---- invariances -----------------------------------------------------------------

def test_global_rigid_transform_leaves_cost_unchanged():
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    c0, planes0 = oracle.voxel_pass(prob, s.pose_init)
    Rg, tg = _rigid(np.random.default_rng(8))
    moved = s.pose_init.copy()
    for j in range(s.n_scans):
        R = s.pose_init[j, :9].reshape(3, 3)
        moved[j, :9] = (Rg @ R).ravel()
        moved[j, 9:] = Rg @ s.pose_init[j, 9:] + tg
    c1, planes1 = oracle.voxel_pass(prob, moved)
    assert c1 == pytest.approx(c0, rel=1e-12)
    np.testing.assert_allclose(planes1[:, :3], planes0[:, :3], rtol=1e-8, atol=1e-15)
    np.testing.assert_allclose(np.abs(np.sum(planes1[:, 3:6] * (planes0[:, 3:6] @ Rg.T), 1)), 1.0, atol=1e-9)


def test_observation_order_does_not_change_cost():
    s, pts, po, raw, cen = tiny_scene()
    rng = np.random.default_rng(12)
    perm_vox = rng.permutation(s.n_voxels)
    new_off = [0]
    new_scan = []
    new_agg = []
    for i in perm_vox:
        lo, hi = s.voxel_off[i], s.voxel_off[i + 1]
        idx = rng.permutation(np.arange(lo, hi))
        new_scan.append(s.obs_scan[idx])
        new_agg.append(cen[idx])
        new_off.append(new_off[-1] + hi - lo)
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    prob2 = oracle.ObsProblem(s.n_scans, np.array(new_off), np.concatenate(new_scan), np.concatenate(new_agg))
    c0, _ = oracle.voxel_pass(prob, s.pose_init)
    c1, _ = oracle.voxel_pass(prob2, s.pose_init)
    assert c1 == pytest.approx(c0, rel=1e-13)


# ---- LM ------------------------------------------------------------------------------

def test_lm_accepted_costs_strictly_decrease():
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    lm = oracle.LM(prob, s.pose_init)
    costs = [lm.cost]
    for _ in range(20):
        if lm.step():
            costs.append(lm.cost)
    assert len(costs) > 10
    assert all(b < a for a, b in zip(costs, costs[1:]))
    # scan 0 is held fixed (gauge)
    np.testing.assert_array_equal(lm.poses[0], s.pose_init[0])


def test_noise_free_scene_returns_ground_truth():
    s, pts, po, raw, cen = tiny_scene(noise_sigma=0.0, rot_sigma_deg=0.1, trans_sigma=0.01)
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    lm = oracle.LM(prob, s.pose_init, rel_tol=0.0, max_iters=300)
    lm.solve()
    rot, tr = pose_errors(lm.poses, s.pose_gt)
    assert rot < 1e-6 and tr < 1e-5
    assert lm.cost < 1e-10


def test_lm_rejects_when_damping_solve_fails():
    """A non-positive pivot makes the whole step a rejection (mu grows, poses kept)."""
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    lm = oracle.LM(prob, s.pose_init)
    lm.H[3] = -np.eye(6)  # planted failure, oracle side only
    before = lm.poses.copy()
    mu = lm.mu
    assert not lm.step()
    assert lm.st.solve_failed == 1
    np.testing.assert_array_equal(lm.poses, before)
    assert lm.mu == pytest.approx(2.0 * mu)


# ---- LM rule: predicted reduction and Nielsen damping update (Sec. IV-C, Algorithm 2
# PredResReduction / Adjust; the rule of Madsen, Nielsen & Tingleff 2004) ---------------
#
# The predicted reduction L is the decrease of the quadratic model of the MM surrogate,
# and the surrogate (Eq. 3, fixed-plane form) is evaluated here by brute force over the
# raw points (oracle.surrogate_points, pinned above), so L is checked against the
# function it models rather than against its own formula.

def _surrogate(s, po, pts, poses, planes_l):
    return oracle.surrogate_points(s.voxel_off, s.obs_scan, po, pts, poses, planes_l)


def _translation_only(lm):
    """Decouple the rotation block from g and H (oracle state, CPU): the damped
    solve then returns a zero rotation increment, so the trial pose moves only
    t, along which the surrogate is exactly quadratic."""
    lm.g[:, :3] = 0.0
    lm.H[:, :3, 3:] = 0.0
    lm.H[:, 3:, :3] = 0.0


def _translation_step(lm, s):
    """The trial poses of a translation-only step, from numpy's solver:
    (H_tt + mu diag(H_tt)) dt = -g_t per scan, scan 0 (the gauge) fixed."""
    P1 = lm.poses.copy()
    seen = np.bincount(s.obs_scan, minlength=s.n_scans) > 0
    for j in range(1, s.n_scans):
        if not seen[j]:
            continue
        Htt = lm.H[j, 3:, 3:]
        P1[j, 9:] += np.linalg.solve(Htt + lm.mu * np.diag(np.diag(Htt)), -lm.g[j, 3:])
    return P1


def test_lm_prediction_equals_surrogate_decrease_for_translation_steps():
    """Along t the surrogate is a quadratic, so L = c_M(T^l) - c_M(T') to rounding."""
    s, pts, po, raw, cen = tiny_scene()
    lm = oracle.LM(oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen), s.pose_init)
    P0, planes_l = lm.poses.copy(), lm.planes.copy()
    _translation_only(lm)
    expect = _translation_step(lm, s)
    assert lm.step()
    np.testing.assert_array_equal(lm.poses[:, :9], P0[:, :9])  # Exp(0) R = R exactly
    np.testing.assert_allclose(lm.poses[:, 9:], expect[:, 9:], rtol=0, atol=1e-12)
    dec = _surrogate(s, po, pts, P0, planes_l) - _surrogate(s, po, pts, lm.poses, planes_l)
    assert dec > 0
    assert lm.st.last_pred == pytest.approx(dec, rel=1e-10)


def test_lm_prediction_matches_surrogate_to_third_order():
    """For a general increment the model error is O(|D|^3): the third-order
    coefficient err / |D|^3 stays put while the step shrinks by 30x (a wrong
    weight of the quadratic term, or a wrong rotation term of the exact
    Hessian, leaves an O(|D|^2) error, whose coefficient grows as 1/|D|)."""
    from tests._util import rot_angle
    s, pts, po, raw, cen = tiny_scene()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen)
    coef, rel = [], []
    for mu in (30.0, 100.0, 300.0, 1000.0):
        lm = oracle.LM(prob, s.pose_init)
        lm.st.mu = mu
        P0, planes_l = lm.poses.copy(), lm.planes.copy()
        assert lm.step()
        P1 = lm.poses
        d = max(np.hypot(rot_angle(b[:9].reshape(3, 3) @ a[:9].reshape(3, 3).T), np.linalg.norm(b[9:] - a[9:]))
                for a, b in zip(P0, P1))
        dec = _surrogate(s, po, pts, P0, planes_l) - _surrogate(s, po, pts, P1, planes_l)
        err = abs(lm.st.last_pred - dec)
        coef.append(err / d ** 3)
        rel.append(err / dec)
    assert max(coef) < 2.0 * min(coef), coef
    assert rel[-1] < 1e-8, rel


@pytest.mark.parametrize("rho", [0.2, 0.5, 0.75, 0.9, 1.3])
def test_lm_damping_update_follows_nielsen(rho):
    """After an accepted step mu' = mu max(1/3, 1 - (2 rho - 1)^3) and nu = 2, with
    rho = (c - c') / (c_M(T^l) - c_M(T')) formed here: c' by brute force over the
    raw points, the surrogate decrease likewise.  The cost the step starts from is
    set so that the step has the chosen gain ratio."""
    s, pts, po, raw, cen = tiny_scene()
    lm = oracle.LM(oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen), s.pose_init)
    P0, planes_l = lm.poses.copy(), lm.planes.copy()
    _translation_only(lm)
    P1 = _translation_step(lm, s)
    c1, _ = oracle.cost_points(s.voxel_off, s.obs_scan, po, pts, P1)
    L = _surrogate(s, po, pts, P0, planes_l) - _surrogate(s, po, pts, P1, planes_l)
    lm.st.cost = c1 + rho * L
    lm.st.nu = 8.0
    mu = lm.mu
    assert lm.step()
    assert lm.st.last_rho == pytest.approx(rho, rel=1e-8)
    assert lm.mu == pytest.approx(mu * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), rel=1e-8)
    assert lm.nu == 2.0
    assert lm.cost == pytest.approx(c1, rel=1e-12)


def test_lm_rejection_by_cost_raises_damping():
    """c(T') >= c(T) rejects: poses kept, mu *= nu, nu *= 2, twice in a row."""
    s, pts, po, raw, cen = tiny_scene()
    lm = oracle.LM(oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen), s.pose_init)
    P0 = lm.poses.copy()
    _translation_only(lm)
    P1 = _translation_step(lm, s)
    c1, _ = oracle.cost_points(s.voxel_off, s.obs_scan, po, pts, P1)
    lm.st.cost = c1 * (1.0 - 1e-9)
    mu = lm.mu
    assert not lm.step()
    np.testing.assert_array_equal(lm.poses, P0)
    assert lm.mu == pytest.approx(2.0 * mu) and lm.nu == 4.0
    assert lm.st.last_rho < 0
    assert not lm.step()
    assert lm.mu == pytest.approx(8.0 * mu) and lm.nu == 8.0
    assert lm.st.consec_reject == 2
