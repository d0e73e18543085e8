"""Seeded synthetic planar scenes (input synthesis only).

The C source next to this file draws every random number from a counter-based
generator (SplitMix64 output function), so a scene is a pure function of its
parameters and seed, and any range of observations' points can be produced on
its own.  Both the CPU oracle and the CUDA library consume these scenes; this
module holds none of the bundle-adjustment arithmetic.

Workloads (sizes follow the paper's dataset scales, Sec. VI-A/B: >10k poses,
>200M points; the datasets themselves are not used):

* ``tiny``  -- 20 scans, 200 voxels, 5-20 observations per voxel, 50 points per
  observation, 1 m x 1 m patches in a 50 m cube, 1 cm noise, 1 deg / 5 cm
  initial perturbation.
* ``mid``   -- 1,000 scans, 50,000 voxels, 8-40 observations (~1.2M), 100
  points each (~120M), 2 cm noise, 0.5 deg / 10 cm.
* ``city``  -- 10,000 scans, 500,000 voxels, 10-50 observations (~15M), 32
  points each, patch side log-uniform 0.5-4 m, 5% strip voxels, 2 cm noise,
  0.5 deg / 10 cm, a 2 km x 2 km x 50 m slab with scans chosen within 200 m.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scenegen.c")
_HDR = os.path.join(_HERE, "scenegen.h")
_LIB = os.path.join(_HERE, "libscenegen.so")
_lock = threading.Lock()
_lib = None


_GPU_SRC = os.path.join(_HERE, "scenegen_gpu.cu")
_GPU_LIB = os.path.join(_HERE, "libscenegen_gpu.so")
_gpu_lib = None


def build(force: bool = False) -> str:
    """Compile the generator into a shared library beside its source."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(src) > os.path.getmtime(_LIB) for src in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def build_gpu(force: bool = False) -> str:
    """Compile the CUDA point generator (sm_103a) beside its source."""
    import shutil
    stale = (not os.path.exists(_GPU_LIB)) or any(
        os.path.getmtime(src) > os.path.getmtime(_GPU_LIB) for src in (_GPU_SRC, _HDR))
    if force or stale:
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = _GPU_LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC",
                               "-shared", "-o", tmp, _GPU_SRC])
        os.replace(tmp, _GPU_LIB)
    return _GPU_LIB


def _load_gpu():
    global _gpu_lib
    with _lock:
        if _gpu_lib is None:
            lib = ctypes.CDLL(build_gpu())
            lib.sgd_points.restype = ctypes.c_int
            lib.sgd_points.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_double] + [ctypes.c_void_p] * 5 + \
                [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            lib.sgd_points_fast.restype = ctypes.c_int
            lib.sgd_points_fast.argtypes = lib.sgd_points.argtypes
            lib.sgd_job.restype = ctypes.c_int
            lib.sgd_job.argtypes = [ctypes.c_void_p] * 10
            _gpu_lib = lib
    return _gpu_lib


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_scans", ctypes.c_int32),
        ("pts_per_obs", ctypes.c_int32),
        ("n_voxels", ctypes.c_int64),
        ("obs_min", ctypes.c_int32),
        ("obs_max", ctypes.c_int32),
        ("box", ctypes.c_double * 3),
        ("side_min", ctypes.c_double),
        ("side_max", ctypes.c_double),
        ("noise_sigma", ctypes.c_double),
        ("rot_sigma_deg", ctypes.c_double),
        ("trans_sigma", ctypes.c_double),
        ("degenerate_frac", ctypes.c_double),
        ("view_radius", ctypes.c_double),
        ("perturb_scan0", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.sg_create.restype = ctypes.c_void_p
            lib.sg_create.argtypes = [ctypes.POINTER(_Params)]
            lib.sg_destroy.argtypes = [ctypes.c_void_p]
            lib.sg_n_obs.restype = ctypes.c_int64
            lib.sg_n_obs.argtypes = [ctypes.c_void_p]
            lib.sg_n_points.restype = ctypes.c_int64
            lib.sg_n_points.argtypes = [ctypes.c_void_p]
            lib.sg_copy.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 6
            lib.sg_voxel_offsets.restype = ctypes.c_int64
            lib.sg_voxel_offsets.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p]
            lib.sg_points.restype = ctypes.c_int
            lib.sg_points.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_int]
            _lib = lib
    return _lib


@dataclass(frozen=True)
class SceneParams:
    n_scans: int
    n_voxels: int
    obs_min: int
    obs_max: int
    pts_per_obs: int
    box: tuple = (50.0, 50.0, 50.0)
    side_min: float = 1.0
    side_max: float = 1.0
    noise_sigma: float = 0.01
    rot_sigma_deg: float = 1.0
    trans_sigma: float = 0.05
    degenerate_frac: float = 0.0
    view_radius: float = 0.0
    perturb_scan0: bool = False
    seed: int = 0


CONFIGS = {
    "tiny": SceneParams(n_scans=20, n_voxels=200, obs_min=5, obs_max=20, pts_per_obs=50,
                        noise_sigma=0.01, rot_sigma_deg=1.0, trans_sigma=0.05),
    "mid": SceneParams(n_scans=1000, n_voxels=50_000, obs_min=8, obs_max=40, pts_per_obs=100,
                       noise_sigma=0.02, rot_sigma_deg=0.5, trans_sigma=0.10),
    "city": SceneParams(n_scans=10_000, n_voxels=500_000, obs_min=10, obs_max=50, pts_per_obs=32,
                        box=(2000.0, 2000.0, 50.0), side_min=0.5, side_max=4.0, noise_sigma=0.02,
                        rot_sigma_deg=0.5, trans_sigma=0.10, degenerate_frac=0.05, view_radius=200.0),
}
CONFIG_INDEX = {"tiny": 1, "mid": 2, "city": 3}


def config(name: str, rep: int = 0, **overrides) -> SceneParams:
    """Named workload with seed 1000*index + rep and optional field overrides."""
    p = replace(CONFIGS[name], seed=1000 * CONFIG_INDEX[name] + rep)
    return replace(p, **overrides) if overrides else p


@dataclass
class Scene:
    params: SceneParams
    pose_gt: np.ndarray      # (n_scans, 12) float64
    pose_init: np.ndarray    # (n_scans, 12) float64
    plane: np.ndarray        # (n_voxels, 12): centre, normal, e1, e2
    extent: np.ndarray       # (n_voxels, 2)
    voxel_off: np.ndarray    # (n_voxels + 1,) int64
    obs_scan: np.ndarray     # (n_obs,) int32
    _handle: object = field(default=None, repr=False)

    @property
    def n_scans(self) -> int:
        return self.params.n_scans

    @property
    def n_voxels(self) -> int:
        return self.params.n_voxels

    @property
    def n_obs(self) -> int:
        return int(self.obs_scan.shape[0])

    @property
    def n_points(self) -> int:
        return self.n_obs * self.params.pts_per_obs

    def point_offsets(self) -> np.ndarray:
        return np.arange(self.n_obs + 1, dtype=np.int64) * self.params.pts_per_obs

    def points(self, obs_begin: int = 0, obs_end: int | None = None, nthreads: int | None = None,
               out: np.ndarray | None = None) -> np.ndarray:
        """Raw scan-frame points of observations [obs_begin, obs_end), (n, 3) float64."""
        if obs_end is None:
            obs_end = self.n_obs
        n = (obs_end - obs_begin) * self.params.pts_per_obs
        if out is None:
            out = np.empty((n, 3), dtype=np.float64)
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == (n, 3)
        if nthreads is None:
            nthreads = min(32, os.cpu_count() or 1)
        rc = _load().sg_points(self._handle, obs_begin, obs_end, out.ctypes.data, nthreads)
        if rc != 0:
            raise ValueError("bad observation range")
        return out

    def points_device(self, obs_begin: int, obs_end: int, out, stream=None):
        """Points of observations [obs_begin, obs_end) generated on the GPU into
        `out`, a CUDA float64 tensor of shape (n, 3); same streams as points()."""
        import torch
        dev = out.device
        cache = getattr(self, "_dev_cache", None)
        if cache is None or cache[0] != dev:
            obs_voxel = np.repeat(np.arange(self.n_voxels, dtype=np.int32), np.diff(self.voxel_off))
            T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
            cache = (dev, T(self.plane), T(self.extent), T(self.pose_gt), T(self.obs_scan), T(obs_voxel))
            self._dev_cache = cache
        _, plane, extent, pose, oscan, ovox = cache
        n = (obs_end - obs_begin) * self.params.pts_per_obs
        assert out.dtype == torch.float64 and out.is_contiguous() and tuple(out.shape) == (n, 3)
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        rc = _load_gpu().sgd_points(self.params.seed, self.params.pts_per_obs, self.params.noise_sigma,
                                    plane.data_ptr(), extent.data_ptr(), pose.data_ptr(), oscan.data_ptr(),
                                    ovox.data_ptr(), obs_begin, obs_end, out.data_ptr(), s)
        if rc != 0:
            raise RuntimeError(f"scenegen GPU point generation failed (CUDA error {rc})")
        return out

    def close(self):
        if self._handle is not None:
            _load().sg_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cparams(p: SceneParams) -> _Params:
    return _Params(seed=p.seed, n_scans=p.n_scans, pts_per_obs=p.pts_per_obs, n_voxels=p.n_voxels,
                   obs_min=p.obs_min, obs_max=p.obs_max, box=(ctypes.c_double * 3)(*p.box),
                   side_min=p.side_min, side_max=p.side_max, noise_sigma=p.noise_sigma,
                   rot_sigma_deg=p.rot_sigma_deg, trans_sigma=p.trans_sigma,
                   degenerate_frac=p.degenerate_frac, view_radius=p.view_radius,
                   perturb_scan0=int(p.perturb_scan0), reserved=0)


def voxel_offsets(p: SceneParams, out: np.ndarray | None = None) -> np.ndarray:
    """Voxel-major observation offsets of the scene p describes (n_voxels + 1
    int64), from the count stream alone; scenes without a view radius only."""
    if out is None:
        out = np.empty(p.n_voxels + 1, dtype=np.int64)
    assert out.dtype == np.int64 and out.flags.c_contiguous and out.shape == (p.n_voxels + 1,)
    n = _load().sg_voxel_offsets(ctypes.byref(_cparams(p)), out.ctypes.data)
    if n < 0:
        raise ValueError("voxel_offsets needs a scene without a view radius")
    return out


@dataclass
class DeviceScene:
    """A scene without a view radius generated on the GPU (sgd_job): the same
    structure, poses and patches as make_scene(params), as CUDA tensors.
    Everything is queued on the stream given to make_scene_device and is
    ready once that stream reaches it."""
    params: SceneParams
    n_obs: int
    voxel_off: object   # (n_voxels + 1,) int64
    obs_scan: object    # (n_obs,) int32
    obs_voxel: object   # (n_obs,) int32
    pose_gt: object     # (n_scans, 12) float64
    pose_init: object   # (n_scans, 12) float64
    plane: object       # (n_voxels, 12)
    extent: object      # (n_voxels, 2)
    bad: object         # (1,) int32: 1 if the generator met an offset it could not take
    host_off: np.ndarray = field(default=None, repr=False)  # pinned source of voxel_off

    @property
    def n_scans(self) -> int:
        return self.params.n_scans

    @property
    def n_voxels(self) -> int:
        return self.params.n_voxels

    def _points(self, fn, obs_begin, obs_end, out, stream):
        import torch
        n = (obs_end - obs_begin) * self.params.pts_per_obs
        assert out.dtype == torch.float64 and out.is_contiguous() and tuple(out.shape) == (n, 3)
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        rc = fn(self.params.seed, self.params.pts_per_obs, self.params.noise_sigma, self.plane.data_ptr(),
                self.extent.data_ptr(), self.pose_gt.data_ptr(), self.obs_scan.data_ptr(), self.obs_voxel.data_ptr(),
                obs_begin, obs_end, out.data_ptr(), s)
        if rc != 0:
            raise RuntimeError(f"scenegen GPU point generation failed (CUDA error {rc})")
        return out

    def points(self, obs_begin, obs_end, out, stream=None):
        """FP64 points, as Scene.points_device (equal to the host's up to the
        last bits of the math library)."""
        return self._points(_load_gpu().sgd_points, obs_begin, obs_end, out, stream)

    def points_fast(self, obs_begin, obs_end, out, stream=None):
        """Points drawn in FP32 from the same per-observation counters (a few
        micrometres from the FP64 points; see scenegen_gpu.cu)."""
        return self._points(_load_gpu().sgd_points_fast, obs_begin, obs_end, out, stream)


def pinned_voxel_offsets(p: SceneParams):
    """voxel_offsets(p) into pinned host memory (a CPU int64 tensor), ready
    for an asynchronous copy; safe to call from worker threads."""
    import torch
    host_off = torch.empty(p.n_voxels + 1, dtype=torch.int64).pin_memory()
    voxel_offsets(p, host_off.numpy())
    return host_off


def make_scene_device(p: SceneParams, device=None, stream=None, offsets=None) -> DeviceScene:
    """Generate the scene p on the GPU (no view radius; obs_max <= 64).  The
    offsets come from the host's count stream (cheap; pass them precomputed
    by pinned_voxel_offsets as `offsets`), everything else from device
    kernels queued on `stream` (default: the current stream)."""
    import torch
    dev = torch.device("cuda") if device is None else torch.device(device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    host_off = offsets if offsets is not None else pinned_voxel_offsets(p)
    n_obs = int(host_off[-1])
    with torch.cuda.stream(st):
        e = lambda *shape, dt=torch.float64: torch.empty(shape, dtype=dt, device=dev)
        voxel_off = host_off.to(dev, non_blocking=True)
        sc = DeviceScene(p, n_obs, voxel_off, e(max(n_obs, 1), dt=torch.int32)[:n_obs],
                         e(max(n_obs, 1), dt=torch.int32)[:n_obs], e(p.n_scans, 12), e(p.n_scans, 12),
                         e(max(p.n_voxels, 1), 12)[: p.n_voxels], e(max(p.n_voxels, 1), 2)[: p.n_voxels],
                         torch.zeros(1, dtype=torch.int32, device=dev), host_off=host_off)
    cp = _cparams(p)
    rc = _load_gpu().sgd_job(ctypes.byref(cp), sc.voxel_off.data_ptr(), sc.pose_gt.data_ptr(),
                             sc.pose_init.data_ptr(), sc.plane.data_ptr(), sc.extent.data_ptr(),
                             sc.obs_scan.data_ptr(), sc.obs_voxel.data_ptr(), sc.bad.data_ptr(), st.cuda_stream)
    if rc != 0:
        raise RuntimeError(f"scenegen GPU job generation failed ({rc})")
    return sc


def make_scene(p: SceneParams) -> Scene:
    lib = _load()
    cp = _cparams(p)
    h = lib.sg_create(ctypes.byref(cp))
    if not h:
        raise ValueError(f"invalid scene parameters {p}")
    n_obs = lib.sg_n_obs(h)
    pose_gt = np.empty((p.n_scans, 12))
    pose_init = np.empty((p.n_scans, 12))
    plane = np.empty((p.n_voxels, 12))
    extent = np.empty((p.n_voxels, 2))
    voxel_off = np.empty(p.n_voxels + 1, dtype=np.int64)
    obs_scan = np.empty(max(n_obs, 1), dtype=np.int32)[:n_obs]
    lib.sg_copy(h, pose_gt.ctypes.data, pose_init.ctypes.data, plane.ctypes.data, extent.ctypes.data,
                voxel_off.ctypes.data, obs_scan.ctypes.data)
    return Scene(p, pose_gt, pose_init, plane, extent, voxel_off, obs_scan, _handle=h)
