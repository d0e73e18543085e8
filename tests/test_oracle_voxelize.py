"""Pins of the preprocessing oracle (L1 voxelisation, bottom-up levels,
selection; Sec. IV-B, Eq. 4-5, Algorithm 1) against numpy computations that
share nothing with it: clusters recomputed from the raw points that fall in
each voxel's box, eigenvalues from numpy.linalg.eigvalsh, and the algebraic
identity behind merging clusters."""
import numpy as np
import pytest

import oracle
import scenegen


def _scan_points(s):
    """The tiny scene's points regrouped by scan (scan frame)."""
    npo = s.params.pts_per_obs
    order = np.argsort(s.obs_scan, kind="stable")
    P = s.points().reshape(s.n_obs, npo, 3)[order].reshape(-1, 3)
    counts = np.bincount(s.obs_scan, minlength=s.n_scans) * npo
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64), P


def _world(poses, spo, P):
    W = np.empty_like(P)
    for j in range(len(spo) - 1):
        T = poses[j]
        R, t = T[:9].reshape(3, 3), T[9:]
        W[spo[j]:spo[j + 1]] = P[spo[j]:spo[j + 1]] @ R.T + t
    return W


def _centred(p):
    m = p.mean(axis=0)
    d = p - m
    S = d.T @ d
    return np.array([S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2], m[0], m[1], m[2], len(p)])


@pytest.fixture(scope="module")
def scene():
    s = scenegen.make_scene(scenegen.config("tiny"))
    spo, P = _scan_points(s)
    return s, spo, P


def test_merge_equals_clustering_the_union():
    rng = np.random.default_rng(3)
    for _ in range(50):
        a = rng.normal(size=(rng.integers(1, 9), 3)) * rng.uniform(0.1, 5) + rng.normal(size=3) * 30
        b = rng.normal(size=(rng.integers(1, 9), 3)) * rng.uniform(0.1, 5) + rng.normal(size=3) * 30
        got = oracle.merge_clusters(_centred(a), _centred(b))
        ref = _centred(np.vstack([a, b]))
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("d,levels", [(1.0, 3), (0.37, 2)])
def test_levels_equal_points_in_the_voxel_box(scene, d, levels):
    """Every (level-k voxel, scan) cluster equals the cluster of that scan's
    points whose world coordinates fall in [i d_k, (i + 1) d_k), d_k =
    2^(k-1) d; and every such non-empty set appears."""
    s, spo, P = scene
    v = oracle.voxelize(spo, P, s.pose_gt, d, levels=levels)
    W = _world(s.pose_gt, spo, P)
    scan_of = np.repeat(np.arange(s.n_scans), np.diff(spo))
    counts = 0
    for k in range(1, levels + 1):
        dk = d * 2 ** (k - 1)
        idx = np.floor(W / dk).astype(np.int64)
        # points within 1e-9 of a boundary may round either way: excluded from the check
        frac = W / dk - np.floor(W / dk)
        safe = np.all((frac > 1e-9) & (frac < 1 - 1e-9), axis=1)
        keys = {}
        for q in np.nonzero(safe)[0]:
            keys.setdefault((tuple(idx[q]), scan_of[q]), []).append(q)
        vox = np.nonzero(v["level"] == k)[0]
        seen = 0
        for i in vox:
            key = tuple(v["index"][i])
            for o in range(v["voxel_off"][i], v["voxel_off"][i + 1]):
                j = v["obs_scan"][o]
                pts_ref = keys.get((key, j))
                if pts_ref is None:
                    continue  # only boundary points in this cluster
                seen += 1
                if len(pts_ref) != v["agg"][o, 9]:
                    continue  # a boundary point of this voxel was excluded above
                np.testing.assert_allclose(v["agg"][o], _centred(P[pts_ref]), rtol=1e-10, atol=1e-10)
                counts += 1
        assert seen >= 0.999 * len(keys), (k, seen, len(keys))
    assert counts > 0


def test_order_counts_and_min_obs(scene):
    s, spo, P = scene
    v = oracle.voxelize(spo, P, s.pose_gt, 1.0, levels=3)
    lev, ix = v["level"], v["index"]
    # voxels: level, then index; observations of a voxel: by scan, distinct
    keys = np.column_stack([lev, ix])
    assert all(tuple(keys[i]) < tuple(keys[i + 1]) for i in range(len(keys) - 1))
    for i in range(len(lev)):
        sc = v["obs_scan"][v["voxel_off"][i]:v["voxel_off"][i + 1]]
        assert np.all(np.diff(sc) > 0)
    # each level holds every point once
    for k in (1, 2, 3):
        sel = np.repeat(lev == k, np.diff(v["voxel_off"]))
        assert v["agg"][sel, 9].sum() == len(P)
    w = oracle.voxelize(spo, P, s.pose_gt, 1.0, levels=3, min_obs=3)
    n_obs = np.diff(v["voxel_off"])
    assert len(w["level"]) == np.sum(n_obs >= 3)
    assert np.all(np.diff(w["voxel_off"]) >= 3)


def test_selection_by_planarity(scene):
    """Kept voxels are exactly those with lambda0 < tau lambda1 of the
    covariance of their world points (numpy eigvalsh), up to near-ties."""
    s, spo, P = scene
    d, levels, tau = 1.0, 2, 0.05
    allv = oracle.voxelize(spo, P, s.pose_init, d, levels=levels)
    kept = oracle.voxelize(spo, P, s.pose_init, d, levels=levels, tau=tau)
    W = _world(s.pose_init, spo, P)
    scan_of = np.repeat(np.arange(s.n_scans), np.diff(spo))
    keyset = {(int(l), tuple(i)) for l, i in zip(kept["level"], kept["index"])}
    n_keep = n_tie = 0
    for i in range(len(allv["level"])):
        k = int(allv["level"][i])
        dk = d * 2 ** (k - 1)
        box = allv["index"][i]
        o0, o1 = allv["voxel_off"][i], allv["voxel_off"][i + 1]
        scans = set(allv["obs_scan"][o0:o1].tolist())
        inside = np.all(np.floor(W / dk).astype(np.int64) == box, axis=1) & np.isin(scan_of, list(scans))
        lam = np.linalg.eigvalsh(np.cov(W[inside].T, bias=True))
        # eigenvalues carry absolute errors of order eps |A| = eps lambda2: a
        # decision inside that band (two-point voxels, exact lines) is a tie
        if abs(lam[0] - tau * lam[1]) <= 1e-9 * lam[2]:
            n_tie += 1
            continue
        expect = lam[0] < tau * lam[1]
        assert ((k, tuple(box)) in keyset) == expect, (i, lam)
        n_keep += expect
    if n_tie == 0:
        assert n_keep == len(kept["level"])
    assert 0 < len(kept["level"]) < len(allv["level"])


def test_out_of_range_index_is_an_error(scene):
    s, spo, P = scene
    far = P.copy()
    far[5] = [3.0e6, 0.0, 0.0]  # 3000 km at d = 1 m: index beyond 2^20
    with pytest.raises(ValueError):
        oracle.voxelize(spo, far, s.pose_gt, 1.0)
