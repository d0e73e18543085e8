"""Shared helpers for the tests: pose error metrics and small fixtures."""
import numpy as np

import scenegen


def skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def rot_angle(R):
    """Rotation angle of R, accurate for small angles (skew part plus trace)."""
    s = 0.5 * np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    c = 0.5 * (np.trace(R) - 1.0)
    return float(np.arctan2(np.linalg.norm(s), c))


def pose_errors(P, Q):
    """max over scans of the rotation angle of R_P R_Q^T (rad) and of |t_P - t_Q| (m)."""
    P = np.asarray(P).reshape(-1, 12)
    Q = np.asarray(Q).reshape(-1, 12)
    rot = 0.0
    for a, b in zip(P, Q):
        rot = max(rot, rot_angle(a[:9].reshape(3, 3) @ b[:9].reshape(3, 3).T))
    tr = float(np.abs(P[:, 9:] - Q[:, 9:]).max()) if len(P) else 0.0
    return rot, tr


_cache = {}


def tiny_scene(**overrides):
    """The 20-scan / 200-voxel workload (points, clusters), cached per parameters."""
    import oracle
    key = tuple(sorted(overrides.items()))
    if key not in _cache:
        s = scenegen.make_scene(scenegen.config("tiny", **overrides))
        pts = s.points()
        po = s.point_offsets()
        raw = oracle.points_to_raw(po, pts)
        cen = oracle.points_to_centred(po, pts)
        _cache[key] = (s, pts, po, raw, cen)
    return _cache[key]


def random_poses_near(poses, rng, rot_sigma, trans_sigma):
    import oracle
    out = np.empty_like(poses)
    for j, p in enumerate(poses):
        d = np.concatenate([rng.normal(0, rot_sigma, 3), rng.normal(0, trans_sigma, 3)])
        out[j] = oracle.retract(p, d)
    return out
