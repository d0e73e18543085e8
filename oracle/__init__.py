"""CPU oracle for the MM LiDAR bundle-adjustment iteration (test infrastructure).

Plain sequential FP64 C (``mmba_oracle.c``) written from the paper's
formulation: point clusters (Eq. 2), the eigenvalue cost (Eq. 1), the MM
surrogate (Eq. 3) and the residual / Jacobian-Hessian / solver steps of
Algorithm 2 under Levenberg-Marquardt control (Sec. IV-C).  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package; the library never does.  This wrapper only marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mmba_oracle.c")
_HDR = os.path.join(_HERE, "mmba_oracle.h")
_SRCS = (_SRC, os.path.join(_HERE, "voxelize_oracle.c"))
_HDRS = (_HDR, os.path.join(_HERE, "voxelize_oracle.h"))
_LIB = os.path.join(_HERE, "libmmba_oracle.so")
_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no fast-math, no contraction)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in _SRCS + _HDRS)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [("n_scans", ctypes.c_int32), ("pad", ctypes.c_int32), ("n_voxels", _I64),
                ("n_obs", _I64), ("voxel_off", _P), ("obs_scan", _P), ("agg", _P)]


class LMConfig(ctypes.Structure):
    _fields_ = [("mu0", _D), ("rel_tol", _D), ("abs_tol", _D), ("fixed_scan", ctypes.c_int32),
                ("gauss_newton", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("max_consec_reject", ctypes.c_int32)]


class LMState(ctypes.Structure):
    _fields_ = [("cost", _D), ("mu", _D), ("nu", _D), ("last_rho", _D), ("last_pred", _D),
                ("last_trial_cost", _D), ("iters", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("consec_reject", ctypes.c_int32), ("last_accepted", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("solve_failed", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "orc_points_to_raw": (None, [_I64, _P, _P, _P]),
                "orc_points_to_centred": (None, [_I64, _P, _P, _P]),
                "orc_raw_to_centred": (None, [_I64, _P, _P]),
                "orc_eig3": (ctypes.c_int, [_P, _P, _P]),
                "orc_cost_points": (_D, [_I64, _P, _P, _P, _P, _P, _P]),
                "orc_cost_eq1": (_D, [_I64, _P, _P, _P, _P, _P]),
                "orc_voxel_pass": (_D, [_P, _P, _P]),
                "orc_surrogate_eq3": (_D, [_I64, _P, _P, _P, _P, _P, _P]),
                "orc_surrogate_points": (_D, [_I64, _P, _P, _P, _P, _P, _P]),
                "orc_grad_hess": (None, [_P, _P, _P, ctypes.c_int, _P, _P]),
                "orc_ldlt6": (ctypes.c_int, [_P, _P, _P]),
                "orc_exp_so3": (None, [_P, _P]),
                "orc_retract": (None, [_P, _P, _P]),
                "orc_lm_init": (None, [_P, _P, _P, _P, _P, _P, _P]),
                "orc_lm_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
                "orc_lm_solve": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
                "orc_world_point": (None, [_P, _P, _P]),
                "orc_merge_clusters": (None, [_P, _P, _P]),
                "orc_voxelize": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _D, ctypes.c_int32, _D, ctypes.c_int32,
                                                _P]),
                "orc_voxels_free": (None, [_P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


# ---- a0: points -> clusters ------------------------------------------------

def points_to_raw(point_off, pts):
    point_off = _c(point_off, np.int64)
    pts = _c(pts, np.float64)
    n = point_off.shape[0] - 1
    out = np.zeros((n, 10))
    _load().orc_points_to_raw(n, _ptr(point_off), _ptr(pts), _ptr(out))
    return out


def points_to_centred(point_off, pts):
    point_off = _c(point_off, np.int64)
    pts = _c(pts, np.float64)
    n = point_off.shape[0] - 1
    out = np.zeros((n, 10))
    _load().orc_points_to_centred(n, _ptr(point_off), _ptr(pts), _ptr(out))
    return out


def raw_to_centred(raw):
    raw = _c(raw, np.float64)
    out = np.zeros_like(raw)
    _load().orc_raw_to_centred(raw.shape[0], _ptr(raw), _ptr(out))
    return out


def eig3(A6):
    """Cyclic Jacobi on a packed symmetric 3x3 (xx, xy, xz, yy, yz, zz)."""
    A6 = _c(A6, np.float64)
    lam = np.zeros(3)
    V = np.zeros(9)
    sweeps = _load().orc_eig3(_ptr(A6), _ptr(lam), _ptr(V))
    return lam, V.reshape(3, 3), sweeps


# ---- problem container ------------------------------------------------------

@dataclass
class ObsProblem:
    """Voxel-major observations with centred clusters (the oracle's input)."""
    n_scans: int
    voxel_off: np.ndarray   # (n_voxels + 1,) int64
    obs_scan: np.ndarray    # (n_obs,) int32
    agg: np.ndarray         # (n_obs, 10) centred clusters

    def __post_init__(self):
        self.voxel_off = _c(self.voxel_off, np.int64)
        self.obs_scan = _c(self.obs_scan, np.int32)
        self.agg = _c(self.agg, np.float64)
        self._cp = Problem(n_scans=self.n_scans, pad=0, n_voxels=self.n_voxels, n_obs=self.n_obs,
                           voxel_off=_ptr(self.voxel_off), obs_scan=_ptr(self.obs_scan),
                           agg=_ptr(self.agg))

    @property
    def n_voxels(self):
        return self.voxel_off.shape[0] - 1

    @property
    def n_obs(self):
        return self.obs_scan.shape[0]

    @property
    def cptr(self):
        return ctypes.byref(self._cp)


def cost_points(voxel_off, obs_scan, point_off, pts, poses):
    voxel_off, obs_scan = _c(voxel_off, np.int64), _c(obs_scan, np.int32)
    point_off, pts, poses = _c(point_off, np.int64), _c(pts, np.float64), _c(poses, np.float64)
    lam0 = np.zeros(voxel_off.shape[0] - 1)
    c = _load().orc_cost_points(lam0.shape[0], _ptr(voxel_off), _ptr(obs_scan), _ptr(point_off), _ptr(pts),
                                _ptr(poses), _ptr(lam0))
    return c, lam0


def cost_eq1(voxel_off, obs_scan, raw, poses):
    voxel_off, obs_scan = _c(voxel_off, np.int64), _c(obs_scan, np.int32)
    raw, poses = _c(raw, np.float64), _c(poses, np.float64)
    lam0 = np.zeros(voxel_off.shape[0] - 1)
    c = _load().orc_cost_eq1(lam0.shape[0], _ptr(voxel_off), _ptr(obs_scan), _ptr(raw), _ptr(poses), _ptr(lam0))
    return c, lam0


def voxel_pass(prob: ObsProblem, poses):
    """Returns (cost, planes) with planes (n_voxels, 9): lam0..2, u, centroid."""
    poses = _c(poses, np.float64)
    planes = np.zeros((prob.n_voxels, 9))
    c = _load().orc_voxel_pass(prob.cptr, _ptr(poses), _ptr(planes))
    return c, planes


def surrogate_eq3(voxel_off, obs_scan, raw, poses, planes_l, poses_l):
    voxel_off, obs_scan = _c(voxel_off, np.int64), _c(obs_scan, np.int32)
    raw, poses = _c(raw, np.float64), _c(poses, np.float64)
    planes_l, poses_l = _c(planes_l, np.float64), _c(poses_l, np.float64)
    return _load().orc_surrogate_eq3(voxel_off.shape[0] - 1, _ptr(voxel_off), _ptr(obs_scan), _ptr(raw),
                                     _ptr(poses), _ptr(planes_l), _ptr(poses_l))


def surrogate_points(voxel_off, obs_scan, point_off, pts, poses, planes_l):
    voxel_off, obs_scan = _c(voxel_off, np.int64), _c(obs_scan, np.int32)
    point_off, pts = _c(point_off, np.int64), _c(pts, np.float64)
    poses, planes_l = _c(poses, np.float64), _c(planes_l, np.float64)
    return _load().orc_surrogate_points(voxel_off.shape[0] - 1, _ptr(voxel_off), _ptr(obs_scan),
                                        _ptr(point_off), _ptr(pts), _ptr(poses), _ptr(planes_l))


def grad_hess(prob: ObsProblem, poses, planes, gauss_newton=False):
    poses, planes = _c(poses, np.float64), _c(planes, np.float64)
    g = np.zeros((prob.n_scans, 6))
    H = np.zeros((prob.n_scans, 6, 6))
    _load().orc_grad_hess(prob.cptr, _ptr(poses), _ptr(planes), int(bool(gauss_newton)), _ptr(g), _ptr(H))
    return g, H


def ldlt6(A, b):
    A, b = _c(A, np.float64), _c(b, np.float64)
    x = np.zeros(6)
    rc = _load().orc_ldlt6(_ptr(A), _ptr(b), _ptr(x))
    return rc, x


def exp_so3(phi):
    phi = _c(phi, np.float64)
    R = np.zeros(9)
    _load().orc_exp_so3(_ptr(phi), _ptr(R))
    return R.reshape(3, 3)


def retract(pose, delta):
    pose, delta = _c(pose, np.float64), _c(delta, np.float64)
    out = np.zeros(12)
    _load().orc_retract(_ptr(pose), _ptr(delta), _ptr(out))
    return out


def retract_all(poses, deltas):
    return np.stack([retract(p, d) for p, d in zip(poses, deltas)])


# ---- LM ----------------------------------------------------------------------

DEFAULT_MU0 = 1e-4


class LM:
    """Oracle LM solver state: poses, planes, g, H, cost, mu, nu."""

    def __init__(self, prob: ObsProblem, poses, mu0=DEFAULT_MU0, rel_tol=1e-8, abs_tol=0.0, fixed_scan=0,
                 gauss_newton=False, max_iters=200, max_consec_reject=10):
        self.prob = prob
        self.cfg = LMConfig(mu0=mu0, rel_tol=rel_tol, abs_tol=abs_tol, fixed_scan=fixed_scan,
                            gauss_newton=int(bool(gauss_newton)), max_iters=max_iters,
                            max_consec_reject=max_consec_reject)
        self.poses = np.array(poses, dtype=np.float64, order="C").reshape(prob.n_scans, 12)
        self.planes = np.zeros((prob.n_voxels, 9))
        self.g = np.zeros((prob.n_scans, 6))
        self.H = np.zeros((prob.n_scans, 6, 6))
        self.st = LMState()
        _load().orc_lm_init(prob.cptr, ctypes.byref(self.cfg), _ptr(self.poses), _ptr(self.planes),
                            _ptr(self.g), _ptr(self.H), ctypes.byref(self.st))

    def step(self) -> bool:
        return bool(_load().orc_lm_step(self.prob.cptr, ctypes.byref(self.cfg), _ptr(self.poses),
                                        _ptr(self.planes), _ptr(self.g), _ptr(self.H), ctypes.byref(self.st)))

    def solve(self) -> int:
        return _load().orc_lm_solve(self.prob.cptr, ctypes.byref(self.cfg), _ptr(self.poses),
                                    _ptr(self.planes), _ptr(self.g), _ptr(self.H), ctypes.byref(self.st))

    @property
    def cost(self):
        return self.st.cost

    @property
    def mu(self):
        return self.st.mu

    @property
    def nu(self):
        return self.st.nu


# ---- preprocessing: L1 voxelisation, bottom-up levels, selection (Sec. IV-B) --

class _Voxels(ctypes.Structure):
    _fields_ = [("n_voxels", _I64), ("n_obs", _I64), ("voxel_off", _P), ("obs_scan", _P), ("agg", _P),
                ("level", _P), ("index", _P)]


def world_point(pose, p):
    pose, p = _c(pose, np.float64), _c(p, np.float64)
    w = np.zeros(3)
    _load().orc_world_point(_ptr(pose), _ptr(p), _ptr(w))
    return w


def merge_clusters(a, b):
    a, b = _c(a, np.float64), _c(b, np.float64)
    out = np.zeros(10)
    _load().orc_merge_clusters(_ptr(a), _ptr(b), _ptr(out))
    return out


def voxelize(scan_point_off, pts, poses, voxel_size, levels=1, tau=0.0, min_obs=1):
    """Raw scans (points of scan j at scan_point_off[j]..) -> voxel-major
    clusters: dict with voxel_off, obs_scan, agg (centred), level, index."""
    spo = _c(scan_point_off, np.int64)
    pts = _c(pts, np.float64).reshape(-1, 3)
    poses = _c(poses, np.float64).reshape(-1, 12)
    v = _Voxels()
    rc = _load().orc_voxelize(int(spo.shape[0] - 1), _ptr(spo), _ptr(pts), _ptr(poses), float(voxel_size),
                              int(levels), float(tau), int(min_obs), ctypes.byref(v))
    if rc != 0:
        raise ValueError("voxelize failed (index out of range or out of memory)")
    try:
        nv, no = v.n_voxels, v.n_obs

        def arr(ptr, dtype, n, shape):
            if n == 0:
                return np.zeros(shape, dtype=dtype)
            ct = ctypes.POINTER(np.ctypeslib.as_ctypes_type(dtype))
            return np.ctypeslib.as_array(ctypes.cast(ptr, ct), shape=(n,)).reshape(shape).copy()
        return {"voxel_off": arr(v.voxel_off, np.int64, nv + 1, (nv + 1,)),
                "obs_scan": arr(v.obs_scan, np.int32, no, (no,)),
                "agg": arr(v.agg, np.float64, 10 * no, (no, 10)),
                "level": arr(v.level, np.int32, nv, (nv,)),
                "index": arr(v.index, np.int32, 3 * nv, (nv, 3))}
    finally:
        _load().orc_voxels_free(ctypes.byref(v))
