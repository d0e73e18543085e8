"""Continuous batching: a job served alongside others that arrive, run and
leave at other times ends with exactly the poses and cost it reaches when
solved alone, and the server keeps its resident jobs inside the memory
budget."""
import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2608_14266_gb300 as mm
    assert torch.cuda.is_available()
    return mm


def _scenes(n_jobs):
    rng = np.random.default_rng(11)
    out = []
    for k in range(n_jobs):
        n_scans = int(rng.integers(6, 30))
        p = scenegen.SceneParams(n_scans=n_scans, n_voxels=50 * n_scans, obs_min=5, obs_max=30, pts_per_obs=16,
                                 noise_sigma=0.02, rot_sigma_deg=0.5, trans_sigma=0.1, seed=7100 + k)
        s = scenegen.make_scene(p)
        out.append((s, s.point_offsets(), s.points()))
    return out


CFG = dict(max_iters=25, rel_tol=1e-10)


def library_clusters(mm, s, po, pts):
    """Centred clusters formed by the library (ba_aggregate_points)."""
    import torch
    agg = torch.empty((s.n_obs, 10), dtype=torch.float64, device="cuda")
    mm.ba_aggregate_points(torch.from_numpy(po).cuda(), torch.from_numpy(pts).cuda(), agg)
    torch.cuda.synchronize()
    return agg.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_served_equals_alone(mm, precision):
    from paper_2608_14266_gb300.server import Job, Server
    prec = mm.BA_MIXED if precision == "mixed" else mm.BA_FP64
    scenes = _scenes(6)
    chunk = 3
    cen = [library_clusters(mm, s, po, pts) for s, po, pts in scenes]
    alone = []
    for (s, po, pts), agg in zip(scenes, cen):
        ba = mm.BundleAdjuster(precision=prec, **CFG)
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, agg, s.pose_init)
        with mm.Batch() as b:
            b.add(ba)
            b.solve(chunk=chunk)
            assert list(b.done()) == [1]
        alone.append((ba.poses(), ba.cost(), ba.stats()["iters"]))
        ba.close()
    # a budget that holds only the two largest jobs at once
    est = [sum(mm.ba_estimate_bytes(prec, s.n_scans, s.n_voxels, s.n_obs)) for s, _, _ in scenes]
    budget = sum(sorted(est)[-2:])
    srv = Server(budget, chunk=chunk, precision=prec, **CFG)
    order = [3, 0, 5, 1, 4, 2]
    submitted = 0
    max_used = 0
    while submitted < len(order) or not srv.idle:
        if submitted < len(order):  # one arrival per round
            k = order[submitted]
            s = scenes[k][0]
            srv.submit(Job(job_id=k, n_scans=s.n_scans, n_voxels=s.n_voxels, n_obs=s.n_obs,
                           inputs=lambda s=s, agg=cen[k]: (s.voxel_off, s.obs_scan, agg, s.pose_init)))
            submitted += 1
        srv.step()
        max_used = max(max_used, srv.used)
        assert srv.used <= budget
    launches = srv.kernel_launches()
    srv.close()
    assert max_used > 0 and launches > 0 and len(srv.finished) == len(scenes)
    # at most two jobs were resident at once, so some waited in the queue
    assert max(j.admitted for j in srv.finished) > min(j.finished for j in srv.finished)
    for job in srv.finished:
        poses, cost, iters = alone[job.job_id]
        np.testing.assert_array_equal(job.poses, poses)
        assert job.stats["cost"] == cost
        assert job.stats["iters"] == iters


def test_estimate_covers_device_bytes(mm):
    """The admission estimate is an upper bound of what a loaded handle holds."""
    for precision in (mm.BA_FP64, mm.BA_MIXED):
        for s, po, pts in _scenes(3):
            keep, peak = mm.ba_estimate_bytes(precision, s.n_scans, s.n_voxels, s.n_obs)
            ba = mm.BundleAdjuster(precision=precision)
            ba.load_points(s.n_scans, s.voxel_off, s.obs_scan, po, pts, s.pose_init)
            assert ba.device_bytes() <= keep
            ba.close()


def test_server_rejects_and_polls(mm):
    """Admission answers: a job larger than the whole budget is an invalid
    argument; one that does not fit next to the resident jobs waits; unknown
    ids are rejected; a finished job is handed out once."""
    import ctypes
    from paper_2608_14266_gb300 import _lib
    from paper_2608_14266_gb300.server import Job, Server
    s, po, pts = _scenes(1)[0]
    agg = library_clusters(mm, s, po, pts)
    keep, peak = mm.ba_estimate_bytes(mm.BA_MIXED, s.n_scans, s.n_voxels, s.n_obs)
    with Server(keep + peak - 1, chunk=4, **CFG) as srv:
        srv.submit(Job(0, s.n_scans, s.n_voxels, s.n_obs, inputs=lambda: (s.voxel_off, s.obs_scan, agg, s.pose_init)))
        with pytest.raises(mm.BAError) as e:
            srv.step()
        assert e.value.status == 1 and "whole budget" in str(e.value) and srv.used == 0
    with Server(keep + peak, chunk=50, **CFG) as srv:
        for k in range(2):
            srv.submit(Job(k, s.n_scans, s.n_voxels, s.n_obs,
                           inputs=lambda: (s.voxel_off, s.obs_scan, agg, s.pose_init)))
        assert srv.step() != [] and len(srv.resident) == 0 and len(srv.queue) == 1
        first = srv.finished[0]
        done = ctypes.c_int32()
        # already handed out, and an id never issued
        for jid in (first.server_id, 999):
            assert _lib.lib().ba_server_poll(srv.s, jid, ctypes.byref(done), None, None) == 1
        srv.step()
        assert len(srv.finished) == 2
        np.testing.assert_array_equal(srv.finished[0].poses, srv.finished[1].poses)


def test_served_failures_and_cancellation_leave_others_unchanged(mm):
    """Failures injected on the host into a served stream: a job whose input
    source raises, a job with a non-finite cluster (refused by the load's
    validation), and a resident job cancelled mid-solve.  Each is reported
    with its reason, its memory is released, and the other jobs end with the
    bits they reach alone."""
    from paper_2608_14266_gb300.server import Job, Server
    prec = mm.BA_MIXED
    scenes = _scenes(6)
    chunk = 3
    cen = [library_clusters(mm, s, po, pts) for s, po, pts in scenes]
    alone = {}
    for k in (0, 2, 4):
        s = scenes[k][0]
        ba = mm.BundleAdjuster(precision=prec, **CFG)
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen[k], s.pose_init)
        with mm.Batch() as b:
            b.add(ba)
            b.solve(chunk=chunk)
        alone[k] = (ba.poses(), ba.cost(), ba.stats()["iters"])
        ba.close()
    bad = cen[3].copy()
    bad[5, 0] = np.nan

    def source_fails():
        raise RuntimeError("input source failed")

    def inputs(k):
        s = scenes[k][0]
        if k == 1:
            return source_fails
        agg = bad if k == 3 else cen[k]
        return lambda: (s.voxel_off, s.obs_scan, agg, s.pose_init)

    jobs = {k: Job(k, scenes[k][0].n_scans, scenes[k][0].n_voxels, scenes[k][0].n_obs, inputs=inputs(k))
            for k in range(6)}
    with Server(1 << 34, chunk=chunk, precision=prec, **CFG) as srv:
        for k in range(6):
            srv.submit(jobs[k])
        srv.step()
        assert {j.job_id for j in srv.failed} == {1, 3}
        assert "input source failed" in jobs[1].error and "BAError" in jobs[3].error
        assert len(srv.resident) == 4  # 0, 2, 4, 5 are running
        before = srv.used
        srv.cancel(jobs[5])
        assert srv.used < before and jobs[5].error == "cancelled"
        with pytest.raises(ValueError):
            srv.cancel(jobs[5])
        while not srv.idle:
            srv.step()
        assert srv.used == 0
        assert {j.job_id for j in srv.finished} == {0, 2, 4}
        assert {j.job_id for j in srv.failed} == {1, 3, 5}
        for job in srv.finished:
            poses, cost, iters = alone[job.job_id]
            np.testing.assert_array_equal(job.poses, poses)
            assert job.stats["cost"] == cost and job.stats["iters"] == iters


def _device_inputs(torch, side, s, agg):
    """A job's inputs produced on a side stream (copies queued there), as a
    generator feeding the server would produce them."""
    with torch.cuda.stream(side):
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().to("cuda", non_blocking=True)
        return T(s.voxel_off), T(s.obs_scan), T(agg), T(s.pose_init)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_async_admission_equals_alone(mm, precision):
    """Jobs admitted by the library's loader thread, their inputs still being
    produced on a side stream when they are submitted, end with exactly the
    bits they reach solved alone; at most two fit the budget at once."""
    import torch
    from paper_2608_14266_gb300.server import Job, Server
    prec = mm.BA_MIXED if precision == "mixed" else mm.BA_FP64
    scenes = _scenes(6)
    chunk = 3
    cen = [library_clusters(mm, s, po, pts) for s, po, pts in scenes]
    alone = []
    for (s, po, pts), agg in zip(scenes, cen):
        ba = mm.BundleAdjuster(precision=prec, **CFG)
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, agg, s.pose_init)
        with mm.Batch() as b:
            b.add(ba)
            b.solve(chunk=chunk)
        alone.append((ba.poses(), ba.cost(), ba.stats()["iters"]))
        ba.close()
    est = [sum(mm.ba_estimate_bytes(prec, s.n_scans, s.n_voxels, s.n_obs)) for s, _, _ in scenes]
    budget = sum(sorted(est)[-2:])
    side = torch.cuda.Stream()
    srv = Server(budget, chunk=chunk, precision=prec, async_admission=True, input_stream=side, **CFG)
    order = [3, 0, 5, 1, 4, 2]
    submitted, max_used, saw_loading = 0, 0, False
    while submitted < len(order) or not srv.idle:
        if submitted < len(order):
            k = order[submitted]
            s = scenes[k][0]
            srv.submit(Job(job_id=k, n_scans=s.n_scans, n_voxels=s.n_voxels, n_obs=s.n_obs,
                           inputs=lambda s=s, agg=cen[k]: _device_inputs(torch, side, s, agg)))
            submitted += 1
        srv._admit()
        saw_loading = saw_loading or bool(srv.loading)
        srv.step()
        max_used = max(max_used, srv.used)
        assert srv.used <= budget
    srv.close()
    assert saw_loading and len(srv.finished) == len(scenes) and not srv.failed
    for job in srv.finished:
        poses, cost, iters = alone[job.job_id]
        np.testing.assert_array_equal(job.poses, poses)
        assert job.stats["cost"] == cost
        assert job.stats["iters"] == iters


def test_async_admission_failures_and_cancellation(mm):
    """On the asynchronous path: a job whose clusters the load's validation
    refuses is reported with the library's message, a job cancelled while
    being admitted never runs, and the others end with their solo bits; the
    budget returns to zero."""
    import ctypes
    import torch
    from paper_2608_14266_gb300 import _lib
    from paper_2608_14266_gb300.server import Job, Server
    prec = mm.BA_MIXED
    scenes = _scenes(4)
    chunk = 3
    cen = [library_clusters(mm, s, po, pts) for s, po, pts in scenes]
    alone = {}
    for k in (0, 2):
        s = scenes[k][0]
        ba = mm.BundleAdjuster(precision=prec, **CFG)
        ba.load_observations(s.n_scans, s.voxel_off, s.obs_scan, cen[k], s.pose_init)
        with mm.Batch() as b:
            b.add(ba)
            b.solve(chunk=chunk)
        alone[k] = (ba.poses(), ba.cost(), ba.stats()["iters"])
        ba.close()
    bad = cen[1].copy()
    bad[3, 2] = np.inf
    side = torch.cuda.Stream()
    agg = {0: cen[0], 1: bad, 2: cen[2], 3: cen[3]}
    jobs = {k: Job(k, scenes[k][0].n_scans, scenes[k][0].n_voxels, scenes[k][0].n_obs,
                   inputs=lambda k=k: _device_inputs(torch, side, scenes[k][0], agg[k])) for k in range(4)}
    with Server(1 << 34, chunk=chunk, precision=prec, async_admission=True, input_stream=side, **CFG) as srv:
        for k in range(4):
            srv.submit(jobs[k])
        srv._admit()
        assert len(srv.loading) == 4
        srv.cancel(jobs[3])  # pending or being loaded: dropped either way
        assert jobs[3].error == "cancelled"
        state = _lib.lib().ba_server_job_state(srv.s, jobs[3].server_id)
        assert state in (_lib.BA_JOB_UNKNOWN, _lib.BA_JOB_LOADING)
        while not srv.idle:
            srv.step()
        assert srv.used == 0 and _lib.lib().ba_server_loading(srv.s) == 0
        assert {j.job_id for j in srv.finished} == {0, 2}
        assert {j.job_id for j in srv.failed} == {1, 3}
        assert "BA_ERR_INVALID_ARG" in jobs[1].error and "finite" in jobs[1].error
        done = ctypes.c_int32()
        assert _lib.lib().ba_server_poll(srv.s, jobs[1].server_id, ctypes.byref(done), None, None) == 1
        for job in srv.finished:
            poses, cost, iters = alone[job.job_id]
            np.testing.assert_array_equal(job.poses, poses)
            assert job.stats["cost"] == cost and job.stats["iters"] == iters
