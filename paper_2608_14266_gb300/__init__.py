"""GB300-native majorization-minimization LiDAR bundle adjustment.

Python binding of libmmba (C ABI in ``include/ba.h``).  The functions below
carry the C names and only marshal arguments: numpy arrays are passed as host
memory, CUDA torch tensors as device memory.  Every step of the solver runs in
the library's CUDA kernels; importing this package never falls back to a CPU
path (calls raise if the library is not built).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (BA_AGG_CENTRED, BA_AGG_RAW_SUMS, BA_FP64, BA_HESS_EXACT, BA_HESS_GAUSS_NEWTON,
                   BA_MEM_DEVICE, BA_MEM_HOST, BA_MIXED, BaConfig, BaStats)

__all__ = ["BAError", "Batch", "BundleAdjuster", "voxelize", "ba_config_default", "ba_create", "ba_load_observations",
           "ba_load_points", "ba_iterate", "ba_solve", "ba_poses", "ba_cost", "ba_get_stats", "ba_set_state",
           "ba_planes", "ba_gradient", "ba_kernel_launches", "ba_destroy", "ba_last_error",
           "ba_aggregate_points", "ba_profile_enable", "ba_profile_read", "BA_FP64", "BA_MIXED", "BA_HESS_EXACT", "BA_HESS_GAUSS_NEWTON",
           "BA_AGG_RAW_SUMS", "BA_AGG_CENTRED", "BA_MEM_HOST", "BA_MEM_DEVICE", "BaConfig", "BaStats"]


class BAError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status: int, handle=None):
    if status != _lib.BA_OK:
        msg = _lib.lib().ba_last_error(handle)
        raise BAError(status, msg.decode() if msg else "")


def _is_torch_cuda(x) -> bool:
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


class _Arg:
    """A contiguous host (numpy) or device (torch CUDA) array of a fixed dtype."""

    def __init__(self, x, np_dtype):
        if _is_torch_cuda(x):
            import torch
            tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[np_dtype]
            if x.dtype != tdt:
                raise TypeError(f"expected {tdt}, got {x.dtype}")
            self.keep = x.contiguous()
            self.ptr = self.keep.data_ptr()
            self.device = True
            self.shape = tuple(self.keep.shape)
        else:
            self.keep = np.ascontiguousarray(x, dtype=np_dtype)
            self.ptr = self.keep.ctypes.data if self.keep.size else None
            self.device = False
            self.shape = self.keep.shape


def _mem_kind(*args: _Arg) -> int:
    kinds = {a.device for a in args}
    if len(kinds) != 1:
        raise ValueError("inputs must be all host (numpy) or all device (CUDA tensors)")
    return BA_MEM_DEVICE if kinds.pop() else BA_MEM_HOST


def ba_config_default(**overrides) -> BaConfig:
    cfg = BaConfig()
    _lib.lib().ba_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream  # a torch.cuda.Stream
        setattr(cfg, k, v)
    return cfg


def ba_create(cfg: BaConfig | None = None):
    h = ctypes.c_void_p()
    _check(_lib.lib().ba_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h)), None)
    return h


def ba_load_observations(h, n_scans: int, voxel_offsets, obs_scan, agg, poses, agg_form: int = BA_AGG_CENTRED):
    vo, os_, ag, po = (_Arg(voxel_offsets, np.int64), _Arg(obs_scan, np.int32), _Arg(agg, np.float64),
                       _Arg(poses, np.float64))
    mk = _mem_kind(vo, os_, ag, po)
    n_voxels = vo.shape[0] - 1
    n_obs = os_.shape[0]
    if int(np.prod(ag.shape)) != 10 * n_obs or int(np.prod(po.shape)) != 12 * n_scans:
        raise ValueError("agg must hold n_obs x 10 and poses n_scans x 12 values")
    _check(_lib.lib().ba_load_observations(h, n_scans, n_voxels, n_obs, vo.ptr, os_.ptr, ag.ptr, agg_form, po.ptr,
                                           mk), h)


def ba_load_points(h, n_scans: int, voxel_offsets, obs_scan, point_offsets, points, poses):
    vo, os_, pof, pts, po = (_Arg(voxel_offsets, np.int64), _Arg(obs_scan, np.int32), _Arg(point_offsets, np.int64),
                             _Arg(points, np.float64), _Arg(poses, np.float64))
    mk = _mem_kind(vo, os_, pof, pts, po)
    n_voxels = vo.shape[0] - 1
    n_obs = os_.shape[0]
    if pof.shape[0] != n_obs + 1 or int(np.prod(po.shape)) != 12 * n_scans:
        raise ValueError("point_offsets must hold n_obs + 1 values and poses n_scans x 12")
    _check(_lib.lib().ba_load_points(h, n_scans, n_voxels, n_obs, vo.ptr, os_.ptr, pof.ptr, pts.ptr, po.ptr, mk), h)


def ba_iterate(h, n_iters: int, stats: bool = True):
    st = BaStats()
    _check(_lib.lib().ba_iterate(h, n_iters, ctypes.byref(st) if stats else None), h)
    return st.as_dict() if stats else None


def ba_solve(h):
    st = BaStats()
    _check(_lib.lib().ba_solve(h, ctypes.byref(st)), h)
    return st.as_dict()


def ba_get_stats(h):
    st = BaStats()
    _check(_lib.lib().ba_get_stats(h, ctypes.byref(st)), h)
    return st.as_dict()


def ba_poses(h, n_scans: int | None = None, out=None):
    """Current poses; into `out` (numpy or CUDA tensor of n_scans x 12 float64) if given."""
    if out is None:
        if n_scans is None:
            raise ValueError("n_scans or out is required")
        out = np.empty((n_scans, 12))
    o = _Arg(out, np.float64)
    if not o.device and o.keep is not out:
        raise ValueError("out must be a contiguous float64 array")
    _check(_lib.lib().ba_poses(h, o.ptr, BA_MEM_DEVICE if o.device else BA_MEM_HOST), h)
    return out


def ba_cost(h) -> float:
    c = ctypes.c_double()
    _check(_lib.lib().ba_cost(h, ctypes.byref(c)), h)
    return c.value


def ba_set_state(h, poses, mu: float = 0.0, nu: float = 0.0):
    p = _Arg(poses, np.float64)
    _check(_lib.lib().ba_set_state(h, p.ptr, float(mu), float(nu), BA_MEM_DEVICE if p.device else BA_MEM_HOST), h)


def ba_planes(h, n_voxels: int):
    out = np.empty((n_voxels, 9))
    _check(_lib.lib().ba_planes(h, out.ctypes.data, BA_MEM_HOST), h)
    return out


def ba_gradient(h, n_scans: int):
    g = np.empty((n_scans, 6))
    H = np.empty((n_scans, 6, 6))
    _check(_lib.lib().ba_gradient(h, g.ctypes.data, H.ctypes.data, BA_MEM_HOST), h)
    return g, H


def ba_kernel_launches(h) -> int:
    return int(_lib.lib().ba_kernel_launches(h))


def ba_profile_enable(h, enable: bool = True):
    _check(_lib.lib().ba_profile_enable(h, int(bool(enable))), h)


def ba_profile_read(h) -> dict:
    """{kernel kind: (total ms, launches)} of the event-timed launches."""
    out = {}
    for name, kind in _lib.KERNEL_KINDS.items():
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(_lib.lib().ba_profile_read(h, kind, ctypes.byref(ms), ctypes.byref(n)), h)
        out[name] = (ms.value, n.value)
    return out


def ba_destroy(h):
    if h:
        _lib.lib().ba_destroy(h)


def ba_last_error(h=None) -> str:
    m = _lib.lib().ba_last_error(h)
    return m.decode() if m else ""


def ba_aggregate_points(point_offsets, points, out, stream=None):
    """Centred point clusters on the device (CUDA tensors only)."""
    pof, pts, o = _Arg(point_offsets, np.int64), _Arg(points, np.float64), _Arg(out, np.float64)
    if not (pof.device and pts.device and o.device):
        raise ValueError("ba_aggregate_points takes CUDA tensors")
    s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(_lib.lib().ba_aggregate_points(pof.shape[0] - 1, pof.ptr, pts.ptr, o.ptr, s), None)
    return out


def ba_device_bytes(h) -> int:
    return int(_lib.lib().ba_device_bytes(h))


def ba_estimate_bytes(precision: int, n_scans: int, n_voxels: int, n_obs: int):
    """(bytes a loaded handle holds, extra bytes its load needs transiently)."""
    peak = ctypes.c_int64()
    keep = _lib.lib().ba_estimate_bytes(int(precision), int(n_scans), int(n_voxels), int(n_obs), ctypes.byref(peak))
    return int(keep), int(peak.value)


def ba_eval_cost_noalloc(n_scans, voxel_offsets, obs_scan, agg_centred, poses, cost_out, lambda0_out=None,
                         stream=None):
    """Cost of the given poses without any device allocation by the library.

    For callers that cannot allocate device memory at that point (a fixed
    memory budget in an on-vehicle mapping loop, or a host whose allocator
    already holds the GPU memory).  Every argument is a contiguous CUDA tensor
    owned by the caller: voxel_offsets (n_voxels + 1 int64), obs_scan (n_obs
    int32), agg_centred (n_obs x 10 float64), poses (n_scans x 12 float64);
    the result lands in cost_out (at least one float64) and optionally
    lambda0_out (at least n_voxels float64).  Nothing is copied: a
    non-contiguous or wrongly shaped tensor raises instead (a copy would be
    an allocation, and an output copy would never reach the caller).
    Asynchronous on `stream`; calls that overlap on the GPU share the
    library's scratch and must be serialised.
    """
    import torch
    want = {"voxel_offsets": (voxel_offsets, torch.int64), "obs_scan": (obs_scan, torch.int32),
            "agg_centred": (agg_centred, torch.float64), "poses": (poses, torch.float64),
            "cost_out": (cost_out, torch.float64)}
    if lambda0_out is not None:
        want["lambda0_out"] = (lambda0_out, torch.float64)
    for name, (t, dt) in want.items():
        if not _is_torch_cuda(t):
            raise ValueError(f"ba_eval_cost_noalloc: {name} must be a CUDA tensor")
        if t.dtype != dt:
            raise TypeError(f"ba_eval_cost_noalloc: {name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"ba_eval_cost_noalloc: {name} must be contiguous (no copy is made)")
    if voxel_offsets.dim() != 1 or obs_scan.dim() != 1:
        raise ValueError("ba_eval_cost_noalloc: voxel_offsets and obs_scan must be 1-D")
    n_voxels, n_obs = voxel_offsets.shape[0] - 1, obs_scan.shape[0]
    if tuple(agg_centred.shape) != (n_obs, 10):
        raise ValueError(f"ba_eval_cost_noalloc: agg_centred must be ({n_obs}, 10), got {tuple(agg_centred.shape)}")
    if poses.numel() < 12 * int(n_scans):
        raise ValueError(f"ba_eval_cost_noalloc: poses must hold n_scans x 12 = {12 * int(n_scans)} values")
    if cost_out.numel() < 1:
        raise ValueError("ba_eval_cost_noalloc: cost_out must hold one value")
    if lambda0_out is not None and lambda0_out.numel() < n_voxels:
        raise ValueError(f"ba_eval_cost_noalloc: lambda0_out must hold n_voxels = {n_voxels} values")
    s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    status = _lib.lib().ba_eval_cost_noalloc(int(n_scans), n_voxels, n_obs, voxel_offsets.data_ptr(),
                                            obs_scan.data_ptr(), agg_centred.data_ptr(), poses.data_ptr(),
                                            cost_out.data_ptr(),
                                            lambda0_out.data_ptr() if lambda0_out is not None else None, s)
    if status != _lib.BA_OK:
        raise BAError(status, "ba_eval_cost_noalloc")
    return cost_out


class Batch:
    """Steps many loaded BundleAdjuster jobs together (ba_batch_* in include/ba.h)."""

    def __init__(self, stream=None):
        s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        self.b = ctypes.c_void_p()
        _check(_lib.lib().ba_batch_create(s, ctypes.byref(self.b)), None)
        self.jobs = []

    def _check(self, status):
        if status != _lib.BA_OK:
            raise BAError(status, (_lib.lib().ba_batch_last_error(self.b) or b"").decode())

    def add(self, job: "BundleAdjuster"):
        self._check(_lib.lib().ba_batch_add(self.b, job.h))
        self.jobs.append(job)

    def remove(self, job: "BundleAdjuster"):
        self._check(_lib.lib().ba_batch_remove(self.b, job.h))
        self.jobs.remove(job)

    def __len__(self):
        return int(_lib.lib().ba_batch_size(self.b))

    def iterate(self, n: int):
        self._check(_lib.lib().ba_batch_iterate(self.b, int(n)))

    def solve(self, chunk: int = 8, max_rounds: int = 0) -> int:
        active = ctypes.c_int32()
        self._check(_lib.lib().ba_batch_solve(self.b, int(chunk), int(max_rounds), ctypes.byref(active)))
        return active.value

    def done(self) -> np.ndarray:
        out = np.zeros(len(self.jobs), dtype=np.int32)
        if len(self.jobs):
            self._check(_lib.lib().ba_batch_done(self.b, out.ctypes.data))
        return out.astype(bool)

    def kernel_launches(self) -> int:
        return int(_lib.lib().ba_batch_kernel_launches(self.b))

    def profile(self, enable: bool = True):
        """Per-kernel event timing of later iterations (launched without the graph)."""
        self._check(_lib.lib().ba_batch_profile_enable(self.b, int(bool(enable))))

    def profile_read(self) -> dict:
        """{kernel kind: (total ms, launches)} of the event-timed launches."""
        out = {}
        for name, kind in _lib.KERNEL_KINDS.items():
            if name == "decide":
                continue
            ms, n = ctypes.c_double(), ctypes.c_int64()
            self._check(_lib.lib().ba_batch_profile_read(self.b, kind, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    def autotune(self, iters_per_trial: int = 2, passes: int = 2, cache: str | None = None) -> dict:
        """ba_batch_autotune: picks the voxel pass's launch settings on the
        batch's own iterations; returns the candidates, timings and choice.
        With cache (a JSON file path), a choice stored for this device is
        applied without trials, and a new choice is stored under the device's
        name."""
        key = None
        if cache is not None:
            import json
            import os
            import torch
            key = torch.cuda.get_device_name(self.jobs[0].cfg.device if self.jobs else 0)
            if os.path.exists(cache):
                with open(cache) as f:
                    known = json.load(f).get(key)
                if known:
                    self.set_launch(known["min_blocks"], known["prefetch"])
                    return {"candidates": [], "chosen": -1, "passes": 0, "iterations": 0, "cached": known}
        r = _lib.BaTuneReport()
        self._check(_lib.lib().ba_batch_autotune(self.b, int(iters_per_trial), int(passes), ctypes.byref(r)))
        cands = [{"min_blocks": r.min_blocks[k], "prefetch": r.prefetch[k], "ms_per_iter": r.ms_per_iter[k]}
                 for k in range(r.n_candidates)]
        out = {"candidates": cands, "chosen": r.chosen, "passes": r.passes,
               "iterations": r.n_candidates * int(iters_per_trial) * int(passes)}
        if key is not None and r.chosen >= 0:
            import json
            import os
            table = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    table = json.load(f)
            table[key] = {k: cands[r.chosen][k] for k in ("min_blocks", "prefetch")}
            with open(cache, "w") as f:
                json.dump(table, f, indent=1)
        return out

    def set_launch(self, min_blocks: int, prefetch: int):
        """ba_batch_set_launch: apply stored launch settings (results do not depend on them)."""
        self._check(_lib.lib().ba_batch_set_launch(self.b, int(min_blocks), int(prefetch)))

    def close(self):
        if self.b:
            _lib.lib().ba_batch_destroy(self.b)
            self.b = None
            self.jobs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def voxelize(scan_point_off, points, poses, voxel_size, levels=1, tau=0.0, min_obs=1, device=0, stream=None,
             out="host", profile=False, batch_points=0, alpha=0.25):
    """Raw scans -> voxel-major observations (ba_voxelize, include/ba.h).

    Points of scan j are points[scan_point_off[j]:scan_point_off[j+1]] (scan
    frame); inputs are all numpy (host) or all CUDA tensors (device).  Returns
    a dict voxel_off, obs_scan, agg (centred), level, index, as numpy arrays
    (out="host") or CUDA tensors (out="device"), plus the kernel launch count
    and, with profile=True, "stage_ms": device milliseconds per stage.
    batch_points / alpha size the loader's batches (include/ba.h)."""
    spo, pts, T = _Arg(scan_point_off, np.int64), _Arg(points, np.float64), _Arg(poses, np.float64)
    mk = _mem_kind(spo, pts, T)
    cfg = _lib.BaVoxelizeConfig()
    _lib.lib().ba_voxelize_config_default(ctypes.byref(cfg))
    cfg.voxel_size, cfg.levels, cfg.tau, cfg.min_obs, cfg.device = float(voxel_size), int(levels), float(tau), \
        int(min_obs), int(device)
    cfg.profile = 1 if profile else 0
    cfg.batch_points, cfg.alpha = int(batch_points), float(alpha)
    if stream is not None:
        cfg.cuda_stream = stream if isinstance(stream, int) else stream.cuda_stream
    v = ctypes.c_void_p()
    status = _lib.lib().ba_voxelize(ctypes.byref(cfg), spo.shape[0] - 1, spo.ptr, pts.ptr, T.ptr, mk, ctypes.byref(v))
    if status != _lib.BA_OK:
        raise BAError(status, (_lib.lib().ba_voxelize_last_error() or b"").decode())
    try:
        nv, no = ctypes.c_int64(), ctypes.c_int64()
        _lib.lib().ba_voxels_size(v, ctypes.byref(nv), ctypes.byref(no))
        nv, no = nv.value, no.value
        if out == "device":
            import torch
            dev = torch.device("cuda", int(device))
            res = {"voxel_off": torch.empty(nv + 1, dtype=torch.int64, device=dev),
                   "obs_scan": torch.empty(no, dtype=torch.int32, device=dev),
                   "agg": torch.empty((no, 10), dtype=torch.float64, device=dev),
                   "level": torch.empty(nv, dtype=torch.int32, device=dev),
                   "index": torch.empty((nv, 3), dtype=torch.int32, device=dev)}
            ptr = lambda t: t.data_ptr() if t.numel() else None
            kind = BA_MEM_DEVICE
        else:
            res = {"voxel_off": np.empty(nv + 1, np.int64), "obs_scan": np.empty(no, np.int32),
                   "agg": np.empty((no, 10)), "level": np.empty(nv, np.int32), "index": np.empty((nv, 3), np.int32)}
            ptr = lambda a: a.ctypes.data if a.size else None
            kind = BA_MEM_HOST
        status = _lib.lib().ba_voxels_read(v, ptr(res["voxel_off"]), ptr(res["obs_scan"]), ptr(res["agg"]),
                                           ptr(res["level"]), ptr(res["index"]), kind)
        if status != _lib.BA_OK:
            raise BAError(status, (_lib.lib().ba_voxelize_last_error() or b"").decode())
        res["launches"] = int(_lib.lib().ba_voxels_kernel_launches(v))
        res["batches"] = int(_lib.lib().ba_voxels_batches(v))
        if profile:
            ms = ctypes.c_double()
            res["stage_ms"] = {}
            for i, name in enumerate(_lib.VOX_STAGES):
                _lib.lib().ba_voxels_stage_ms(v, i, ctypes.byref(ms))
                res["stage_ms"][name] = ms.value
        return res
    finally:
        _lib.lib().ba_voxels_destroy(v)


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class BundleAdjuster:
    """Owns one library handle; see include/ba.h for the semantics of each call.

    alloc(bytes, stream) -> device pointer (int, 0 on failure) and
    free(ptr, bytes, stream), if given, replace the library's own pool for the
    handle's device memory (e.g. to draw from PyTorch's caching allocator)."""

    def __init__(self, alloc=None, free=None, **cfg):
        self._callbacks = None
        if (alloc is None) != (free is None):
            raise ValueError("alloc and free must be given together")
        if alloc is not None:
            a = ALLOC_FN(lambda n, stream, ctx: alloc(int(n), stream) or None)
            f = FREE_FN(lambda ptr, n, stream, ctx: free(int(ptr), int(n), stream))
            self._callbacks = (a, f)  # kept alive as long as the handle
            cfg["alloc"] = ctypes.cast(a, ctypes.c_void_p)
            cfg["free"] = ctypes.cast(f, ctypes.c_void_p)
        self.cfg = ba_config_default(**cfg)
        self.h = ba_create(self.cfg)
        self.n_scans = 0
        self.n_voxels = 0

    def load_observations(self, n_scans, voxel_offsets, obs_scan, agg, poses, agg_form=BA_AGG_CENTRED):
        ba_load_observations(self.h, n_scans, voxel_offsets, obs_scan, agg, poses, agg_form)
        self.n_scans, self.n_voxels = n_scans, len(voxel_offsets) - 1
        return self

    def load_points(self, n_scans, voxel_offsets, obs_scan, point_offsets, points, poses):
        ba_load_points(self.h, n_scans, voxel_offsets, obs_scan, point_offsets, points, poses)
        self.n_scans, self.n_voxels = n_scans, len(voxel_offsets) - 1
        return self

    def iterate(self, n=1, stats=True):
        return ba_iterate(self.h, n, stats)

    def solve(self):
        return ba_solve(self.h)

    def poses(self, out=None):
        return ba_poses(self.h, self.n_scans, out)

    def cost(self):
        return ba_cost(self.h)

    def stats(self):
        return ba_get_stats(self.h)

    def set_state(self, poses, mu=0.0, nu=0.0):
        ba_set_state(self.h, poses, mu, nu)

    def planes(self):
        return ba_planes(self.h, self.n_voxels)

    def gradient(self):
        return ba_gradient(self.h, self.n_scans)

    def kernel_launches(self):
        return ba_kernel_launches(self.h)

    def device_bytes(self):
        return ba_device_bytes(self.h)

    def profile(self, enable=True):
        ba_profile_enable(self.h, enable)

    def profile_read(self):
        return ba_profile_read(self.h)

    # voxel-sharded solve (ba_shard_* in include/ba.h)
    def shard_partials(self):
        """(g, H partials as (n_scans, 27) float64, cost partial) at the current poses."""
        gH = np.empty((self.n_scans, 27))
        c = ctypes.c_double()
        _check(_lib.lib().ba_shard_partials(self.h, gH.ctypes.data, ctypes.byref(c), BA_MEM_HOST), self.h)
        return gH, c.value

    def shard_set_totals(self, gH_total, cost_total):
        a = _Arg(gH_total, np.float64)
        if int(np.prod(a.shape)) != 27 * self.n_scans:
            raise ValueError("gH_total must hold n_scans x 27 values")
        _check(_lib.lib().ba_shard_set_totals(self.h, a.ptr, float(cost_total),
                                              BA_MEM_DEVICE if a.device else BA_MEM_HOST), self.h)

    def shard_trial(self) -> float:
        c = ctypes.c_double()
        _check(_lib.lib().ba_shard_trial(self.h, ctypes.byref(c)), self.h)
        return c.value

    def shard_decide(self, trial_cost_total) -> bool:
        acc = ctypes.c_int32()
        _check(_lib.lib().ba_shard_decide(self.h, float(trial_cost_total), ctypes.byref(acc)), self.h)
        return bool(acc.value)

    def close(self):
        if self.h:
            ba_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
