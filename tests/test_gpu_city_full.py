"""Parity at the full city size the bench times (10,000 scans, 500,000
voxels, ~15M clusters), in both precisions, on outputs the oracle can
compute exactly: every voxel's smallest eigenvalue and the cost (the
oracle's full voxel pass), g and H of sampled scans (the oracle on the
sub-problem of every voxel those scans observe, which holds all their
terms), and one full-size iteration's poses of those scans (the oracle's
damped solve and retraction from its own g, H)."""
import numpy as np
import pytest

import oracle
import scenegen
from tests._util import pose_errors

pytestmark = pytest.mark.gpu

# (cost rel, per-voxel lambda rel, g/H rel to the scan's max, rot, trans)
TOL = {"fp64": (1e-10, 1e-9, 1e-9, 1e-9, 1e-8), "mixed": (1e-6, 5e-6, 1e-5, 1e-6, 1e-5)}


@pytest.fixture(scope="module")
def city():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2608_14266_gb300 as mm
    s = scenegen.make_scene(scenegen.config("city"))
    npo = s.params.pts_per_obs
    dev = torch.device("cuda")
    agg = torch.empty((s.n_obs, 10), dtype=torch.float64, device=dev)
    chunk = 1 << 20
    buf = torch.empty((chunk * npo, 3), dtype=torch.float64, device=dev)
    po = torch.arange(chunk + 1, dtype=torch.int64, device=dev) * npo
    for o0 in range(0, s.n_obs, chunk):
        o1 = min(s.n_obs, o0 + chunk)
        pts = buf[: (o1 - o0) * npo]
        s.points_device(o0, o1, pts)
        mm.ba_aggregate_points(po[: o1 - o0 + 1], pts, agg[o0:o1])
    del buf
    torch.cuda.synchronize()
    agg_h = agg.cpu().numpy()
    prob = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, agg_h)
    c0, planes0 = oracle.voxel_pass(prob, s.pose_init)
    return mm, s, agg, agg_h, prob, c0, planes0


def _subproblem(s, agg_h, scans):
    """The voxels observed by any of `scans`, with all their observations."""
    vo = s.voxel_off
    hit = np.isin(s.obs_scan, scans)
    vox = np.unique(np.searchsorted(vo, np.flatnonzero(hit), side="right") - 1)
    cnt = np.diff(vo)[vox]
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    idx = np.repeat(vo[vox], cnt) + (np.arange(int(off[-1])) - np.repeat(off[:-1], cnt))
    return vox, oracle.ObsProblem(s.n_scans, off, s.obs_scan[idx], agg_h[idx])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_city_full_size_sampled_parity(city, precision):
    import torch
    mm, s, agg, agg_h, prob, c0, planes0 = city
    c_tol, lam_tol, gh_tol, rot_tol, tr_tol = TOL[precision]
    prec = mm.BA_MIXED if precision == "mixed" else mm.BA_FP64
    dev = torch.device("cuda")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    with mm.BundleAdjuster(precision=prec) as ba:
        ba.load_observations(s.n_scans, T(s.voxel_off), T(s.obs_scan), agg, T(s.pose_init))
        assert ba.cost() == pytest.approx(c0, rel=c_tol)
        lam = ba.planes()[:, 0]
        rel = np.abs(lam - planes0[:, 0]) / planes0[:, 0]
        assert rel.max() < lam_tol, (rel.max(), int(rel.argmax()))
        # g, H of sampled scans from the sub-problem that holds all their terms
        rng = np.random.default_rng(3)
        scans = np.sort(rng.choice(np.arange(1, s.n_scans), 6, replace=False))
        vox, sub = _subproblem(s, agg_h, scans)
        g_ref, H_ref = oracle.grad_hess(sub, s.pose_init, planes0[vox])
        g, H = ba.gradient()
        for j in scans:
            np.testing.assert_allclose(g[j], g_ref[j], rtol=0, atol=gh_tol * np.abs(g_ref[j]).max())
            np.testing.assert_allclose(H[j], H_ref[j], rtol=0, atol=gh_tol * np.abs(H_ref[j]).max())
        # one iteration at full size: the sampled scans' steps
        st = ba.iterate(1)
        assert st["last_accepted"]
        P = ba.poses()
        mu0 = oracle.DEFAULT_MU0
        expect = np.empty((len(scans), 12))
        for k, j in enumerate(scans):
            A = H_ref[j] + mu0 * np.diag(np.diag(H_ref[j]))
            rc, d = oracle.ldlt6(A, -g_ref[j])
            assert rc == 0
            expect[k] = oracle.retract(s.pose_init[j], d)
        r, t = pose_errors(P[scans], expect)
        assert r < rot_tol and t < tr_tol, (r, t)
        # the accepted cost is the cost at the GPU's new poses
        c1, _ = oracle.voxel_pass(prob, P)
        assert st["cost"] == pytest.approx(c1, rel=c_tol)
