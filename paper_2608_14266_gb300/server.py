"""Continuous-batching bundle-adjustment server (binding of ba_server_* in
include/ba.h).

Jobs (independent BA problems: submaps, sessions) arrive over time.  The
library admits a job when the device bytes of the resident jobs plus the
job's upper estimate fit in the memory budget, keeps every admitted job's
clusters, poses and LM state resident on the GPU, and steps all resident jobs
together (one launch per kernel kind per iteration over a device job table).
A job leaves at the end of the step in which its own stopping rule fired; its
poses are copied to host memory and its device memory is released, so waiting
jobs fit again.  A job's result does not depend on which other jobs shared
its steps.

This module only marshals: it keeps the arrival queue (jobs the library
answered "does not fit now"), prepares a job's inputs when the library says
it fits, and collects finished jobs.  All arithmetic runs in the library.

With async_admission=True a job that fits is handed to the library's loader
thread (ba_server_submit_async): its inputs may still be in production on
`input_stream` (e.g. generated there by GPU kernels) when it is submitted,
and its load and set-up run on a stream of their own while this thread keeps
stepping the resident jobs; the job joins them at the first step after its
load finished.  The inputs are kept alive until the library no longer reads
them.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field
from typing import Callable

import numpy as np

from . import BA_AGG_CENTRED, BA_MIXED, BAError, _Arg, _lib, _mem_kind, ba_config_default
from ._lib import BaJobDesc, BaStats


@dataclass
class Job:
    """inputs() returns (voxel_offsets, obs_scan, agg_centred, poses): all
    numpy arrays (host) or all CUDA tensors (device); it is called once, when
    the job is admitted."""
    job_id: int
    n_scans: int
    n_voxels: int
    n_obs: int
    inputs: Callable[[], tuple]
    arrival: float = 0.0
    admitted: float | None = None
    finished: float | None = None
    poses: np.ndarray | None = None
    stats: dict | None = None
    error: str | None = None  # set when the job failed (its inputs, or the library refused them)
    server_id: int = field(default=0, repr=False)
    keep: object = field(default=None, repr=False)  # inputs held while the library loads them

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival


class Server:
    """mem_budget: device bytes the resident jobs may hold.  chunk: LM
    iterations per step.  Remaining keyword arguments configure every job's
    handle (precision, rel_tol, max_iters, cuda_stream, ...)."""

    def __init__(self, mem_budget: int, chunk: int = 4, clock=time.perf_counter, async_admission: bool = False,
                 input_stream=None, loaders: int = 3, **cfg):
        cfg.setdefault("precision", BA_MIXED)
        self.cfg = ba_config_default(**cfg)
        self.chunk = int(chunk)
        self.clock = clock
        self.async_admission = bool(async_admission)
        self.input_stream = None if input_stream is None else (
            input_stream if isinstance(input_stream, int) else input_stream.cuda_stream)
        self.loading: list[Job] = []
        self.dropping: list[Job] = []  # cancelled while loading; inputs held until the load returns
        self.s = ctypes.c_void_p()
        status = _lib.lib().ba_server_create(ctypes.byref(self.cfg), int(mem_budget), ctypes.byref(self.s))
        if status != _lib.BA_OK:
            raise BAError(status, "ba_server_create")
        self._check(_lib.lib().ba_server_set_loaders(self.s, int(loaders)))
        self.queue: collections.deque[Job] = collections.deque()
        self.resident: list[Job] = []
        self.finished: list[Job] = []
        self.failed: list[Job] = []  # jobs whose inputs failed or were refused; the others carry on

    def _check(self, status):
        if status != _lib.BA_OK:
            raise BAError(status, (_lib.lib().ba_server_last_error(self.s) or b"").decode())

    # -- admission ---------------------------------------------------------
    def submit(self, job: Job) -> None:
        """Queue a job; it is loaded at the next step that has room for it."""
        self.queue.append(job)

    def _admit(self) -> int:
        L = _lib.lib()
        n = 0
        while self.queue:
            job = self.queue[0]
            if not L.ba_server_fits(self.s, job.n_scans, job.n_voxels, job.n_obs):
                if self.resident or self.loading:
                    break
                # nothing resident and still no room: the library reports why (too large for the budget)
                self.queue.popleft()
                desc = BaJobDesc(job.n_scans, job.n_voxels, job.n_obs, None, None, None, BA_AGG_CENTRED, None, 0)
                self._check(L.ba_server_submit(self.s, ctypes.byref(desc), ctypes.byref(ctypes.c_uint64())))
                raise AssertionError("unreachable")
            self.queue.popleft()
            try:
                vo, os_, ag, po = job.inputs()
                a = (_Arg(vo, np.int64), _Arg(os_, np.int32), _Arg(ag, np.float64), _Arg(po, np.float64))
                desc = BaJobDesc(job.n_scans, job.n_voxels, job.n_obs, a[0].ptr, a[1].ptr, a[2].ptr,
                                 BA_AGG_CENTRED, a[3].ptr, _mem_kind(*a))
                jid = ctypes.c_uint64()
                if self.async_admission:
                    self._check(L.ba_server_submit_async(self.s, ctypes.byref(desc), self.input_stream,
                                                         ctypes.byref(jid)))
                else:
                    self._check(L.ba_server_submit(self.s, ctypes.byref(desc), ctypes.byref(jid)))
            except Exception as exc:  # a failed job is reported, the stream goes on
                job.error = f"{type(exc).__name__}: {exc}"
                job.finished = self.clock()
                self.failed.append(job)
                continue
            job.server_id = jid.value
            job.admitted = self.clock()
            if self.async_admission:
                job.keep = a
                self.loading.append(job)
            else:
                self.resident.append(job)
            n += 1
        return n

    def _settle_loading(self) -> None:
        """Jobs whose asynchronous load has returned: resident, or failed."""
        L = _lib.lib()
        for job in list(self.loading):
            state = L.ba_server_job_state(self.s, job.server_id)
            if state == _lib.BA_JOB_LOADING:
                continue
            job.keep = None
            self.loading.remove(job)
            if state == _lib.BA_JOB_FAILED:
                done = ctypes.c_int32()
                status = L.ba_server_poll(self.s, job.server_id, ctypes.byref(done), None, None)
                job.error = f"BAError: {_lib.STATUS_NAMES.get(status, status)}: " + \
                    (L.ba_server_last_error(self.s) or b"").decode()
                job.finished = self.clock()
                self.failed.append(job)
            else:
                self.resident.append(job)

    # -- stepping -----------------------------------------------------------
    def step(self) -> list[Job]:
        """Admit what fits, run one step, collect retired jobs; returns them."""
        self._admit()
        if not self.resident and not self.loading and not self.dropping:
            return []
        L = _lib.lib()
        n_res, n_ret = ctypes.c_int32(), ctypes.c_int32()
        self._check(L.ba_server_step(self.s, self.chunk, ctypes.byref(n_res), ctypes.byref(n_ret)))
        if self.loading:
            self._settle_loading()
        for job in list(self.dropping):
            if L.ba_server_job_state(self.s, job.server_id) != _lib.BA_JOB_LOADING:
                job.keep = None
                self.dropping.remove(job)
        out = []
        if n_ret.value:
            now = self.clock()
            done = ctypes.c_int32()
            st = BaStats()
            for job in list(self.resident):
                poses = np.empty((job.n_scans, 12), dtype=np.float64)
                self._check(L.ba_server_poll(self.s, job.server_id, ctypes.byref(done), poses.ctypes.data,
                                             ctypes.byref(st)))
                if not done.value:
                    continue
                job.poses, job.stats, job.finished = poses, st.as_dict(), now
                self.resident.remove(job)
                self.finished.append(job)
                out.append(job)
        return out

    def cancel(self, job: Job) -> None:
        """Withdraw a queued or resident job (a resident one leaves the batch
        at once and its memory is released)."""
        if job in self.queue:
            self.queue.remove(job)
        elif job in self.resident:
            self._check(_lib.lib().ba_server_cancel(self.s, job.server_id))
            self.resident.remove(job)
        elif job in self.loading:
            self._check(_lib.lib().ba_server_cancel(self.s, job.server_id))
            self.loading.remove(job)
            # the loader thread may be reading its inputs right now: keep them
            # until the library has let go of the job
            self.dropping.append(job)
        else:
            raise ValueError(f"job {job.job_id} is neither queued nor resident")
        job.error = "cancelled"
        job.finished = self.clock()
        self.failed.append(job)

    @property
    def used(self) -> int:
        return int(_lib.lib().ba_server_bytes_in_use(self.s))

    @property
    def idle(self) -> bool:
        return not self.queue and not self.resident and not self.loading and not self.dropping

    def kernel_launches(self) -> int:
        return int(_lib.lib().ba_server_kernel_launches(self.s))

    def close(self):
        if self.s:
            _lib.lib().ba_server_destroy(self.s)
            self.s = None
            self.resident = []
            for job in self.loading + self.dropping:  # the loader thread has stopped
                job.keep = None
            self.loading, self.dropping = [], []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def latency_summary(jobs: list[Job]) -> dict:
    lat = np.array([j.latency for j in jobs if j.latency is not None])
    if lat.size == 0:
        return {"p50_s": None, "p99_s": None, "mean_s": None, "max_s": None}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
