"""ctypes declarations for libmmba.so (the C ABI of include/ba.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# MMBA_CHECKED=1 loads the checked variant (index checks in the kernels, see
# build.build(checked=True)); it is built on request, never implied
LIB_PATH = os.path.join(HERE, "libmmba_checked.so" if os.environ.get("MMBA_CHECKED") == "1" else "libmmba.so")

BA_OK = 0
STATUS_NAMES = {0: "BA_OK", 1: "BA_ERR_INVALID_ARG", 2: "BA_ERR_OOM", 3: "BA_ERR_CUDA", 4: "BA_ERR_STATE",
                5: "BA_ERR_NUMERIC", 6: "BA_ERR_TIMEOUT", 7: "BA_ERR_CAPACITY"}
BA_FP64, BA_MIXED = 0, 1
BA_HESS_EXACT, BA_HESS_GAUSS_NEWTON = 0, 1
BA_MEM_HOST, BA_MEM_DEVICE = 0, 1
BA_AGG_RAW_SUMS, BA_AGG_CENTRED = 0, 1
BA_JOB_UNKNOWN, BA_JOB_LOADING, BA_JOB_RESIDENT, BA_JOB_FINISHED, BA_JOB_FAILED = -1, 0, 1, 2, 3

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double


class BaConfig(ctypes.Structure):
    _fields_ = [("precision", _I32), ("max_iters", _I32), ("rel_tol", _D), ("abs_tol", _D), ("mu0", _D),
                ("fixed_scan", _I32), ("hessian_mode", _I32), ("max_consec_reject", _I32), ("device", _I32),
                ("cuda_stream", _P), ("alloc", _P), ("free", _P), ("alloc_ctx", _P)]


class BaStats(ctypes.Structure):
    _fields_ = [("cost", _D), ("cost_before", _D), ("mu", _D), ("nu", _D), ("last_rho", _D), ("last_pred", _D),
                ("last_trial_cost", _D), ("iters", _I32), ("accepted", _I32), ("consec_reject", _I32),
                ("last_accepted", _I32), ("converged", _I32), ("solve_failed", _I32),
                ("iters_this_call", _I32), ("reserved", _I32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class BaVoxelizeConfig(ctypes.Structure):
    _fields_ = [("voxel_size", _D), ("levels", _I32), ("tau", _D), ("min_obs", _I32), ("device", _I32),
                ("cuda_stream", _P), ("profile", _I32), ("batch_points", _I64), ("alpha", _D)]


class BaTuneReport(ctypes.Structure):
    _fields_ = [("n_candidates", _I32), ("chosen", _I32), ("passes", _I32), ("min_blocks", _I32 * 16),
                ("prefetch", _I32 * 16), ("ms_per_iter", _D * 16)]


class BaJobDesc(ctypes.Structure):
    _fields_ = [("n_scans", _I32), ("n_voxels", _I64), ("n_obs", _I64), ("voxel_offsets", _P), ("obs_scan", _P),
                ("agg", _P), ("agg_form", _I32), ("poses", _P), ("mem_kind", _I32)]


_SIGNATURES = {
    "ba_config_default": (None, [_P]),
    "ba_create": (_I32, [_P, _P]),
    "ba_load_observations": (_I32, [_P, _I32, _I64, _I64, _P, _P, _P, _I32, _P, _I32]),
    "ba_load_points": (_I32, [_P, _I32, _I64, _I64, _P, _P, _P, _P, _P, _I32]),
    "ba_iterate": (_I32, [_P, _I32, _P]),
    "ba_solve": (_I32, [_P, _P]),
    "ba_poses": (_I32, [_P, _P, _I32]),
    "ba_cost": (_I32, [_P, _P]),
    "ba_get_stats": (_I32, [_P, _P]),
    "ba_set_state": (_I32, [_P, _P, _D, _D, _I32]),
    "ba_planes": (_I32, [_P, _P, _I32]),
    "ba_gradient": (_I32, [_P, _P, _P, _I32]),
    "ba_kernel_launches": (_I64, [_P]),
    "ba_destroy": (None, [_P]),
    "ba_last_error": (ctypes.c_char_p, [_P]),
    "ba_status_string": (ctypes.c_char_p, [_I32]),
    "ba_aggregate_points": (_I32, [_I64, _P, _P, _P, _P]),
    "ba_profile_enable": (_I32, [_P, _I32]),
    "ba_profile_read": (_I32, [_P, _I32, _P, _P]),
    "ba_eval_cost_noalloc": (_I32, [_I32, _I64, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "ba_batch_create": (_I32, [_P, _P]),
    "ba_batch_add": (_I32, [_P, _P]),
    "ba_batch_remove": (_I32, [_P, _P]),
    "ba_batch_size": (_I32, [_P]),
    "ba_batch_iterate": (_I32, [_P, _I32]),
    "ba_batch_solve": (_I32, [_P, _I32, _I32, _P]),
    "ba_batch_done": (_I32, [_P, _P]),
    "ba_batch_destroy": (None, [_P]),
    "ba_batch_last_error": (ctypes.c_char_p, [_P]),
    "ba_batch_kernel_launches": (_I64, [_P]),
    "ba_server_create": (_I32, [_P, _I64, _P]),
    "ba_server_submit": (_I32, [_P, _P, _P]),
    "ba_server_step": (_I32, [_P, _I32, _P, _P]),
    "ba_server_poll": (_I32, [_P, ctypes.c_uint64, _P, _P, _P]),
    "ba_server_fits": (_I32, [_P, _I32, _I64, _I64]),
    "ba_server_bytes_in_use": (_I64, [_P]),
    "ba_server_resident": (_I32, [_P]),
    "ba_server_kernel_launches": (_I64, [_P]),
    "ba_server_last_error": (ctypes.c_char_p, [_P]),
    "ba_server_destroy": (None, [_P]),
    "ba_server_cancel": (_I32, [_P, ctypes.c_uint64]),
    "ba_server_submit_async": (_I32, [_P, _P, _P, _P]),
    "ba_batch_profile_enable": (_I32, [_P, _I32]),
    "ba_shard_partials": (_I32, [_P, _P, _P, _I32]),
    "ba_shard_set_totals": (_I32, [_P, _P, _D, _I32]),
    "ba_shard_trial": (_I32, [_P, _P]),
    "ba_shard_decide": (_I32, [_P, _D, _P]),
    "ba_batch_profile_read": (_I32, [_P, _I32, _P, _P]),
    "ba_server_job_state": (_I32, [_P, ctypes.c_uint64]),
    "ba_server_loading": (_I32, [_P]),
    "ba_server_set_loaders": (_I32, [_P, _I32]),
    "ba_check_bounded_wait": (_I32, [_I32, _I32]),
    "ba_release_cached_memory": (_I32, [_I32]),
    "ba_check_conversions": (_I32, [_I32, _I64, ctypes.c_uint64, _P]),
    "ba_batch_autotune": (_I32, [_P, _I32, _I32, _P]),
    "ba_batch_set_launch": (_I32, [_P, _I32, _I32]),
    "ba_voxelize_config_default": (None, [_P]),
    "ba_voxelize": (_I32, [_P, _I32, _P, _P, _P, _I32, _P]),
    "ba_voxels_size": (_I32, [_P, _P, _P]),
    "ba_voxels_read": (_I32, [_P, _P, _P, _P, _P, _P, _I32]),
    "ba_voxels_kernel_launches": (_I64, [_P]),
    "ba_voxels_stage_ms": (_I32, [_P, _I32, _P]),
    "ba_voxels_batches": (_I64, [_P]),
    "ba_voxelize_last_error": (ctypes.c_char_p, []),
    "ba_voxels_destroy": (None, [_P]),
    "ba_device_bytes": (_I64, [_P]),
    "ba_estimate_bytes": (_I64, [_I32, _I32, _I64, _I64, _P]),
}
BA_NOALLOC_MAX_VOXELS = 8388608
BA_KERNEL_VOXEL_PASS, BA_KERNEL_SCAN_PASS, BA_KERNEL_SOLVE, BA_KERNEL_DECIDE = 0, 1, 2, 3
VOX_STAGES = ("keys", "sort", "runs", "cluster_pass", "cluster_finish", "levels", "select", "emit", "merge")
KERNEL_KINDS = {"voxel_pass": 0, "scan_pass": 1, "solve": 2, "decide": 3}

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: the CUDA library must be built first "
                    "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(handle, name)
                f.restype = res
                f.argtypes = args
            _lib = handle
    return _lib


def declared_symbols(header: str) -> list[str]:
    """Names of the functions declared in a C header (for export checks)."""
    import re
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z0-9_]+)\s*\(", text)) - {"ba_alloc_fn", "ba_free_fn"})
