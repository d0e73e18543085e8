"""Batched execution: many jobs stepped together give exactly the results of
each job run alone (every block of a batched launch belongs to one job and
does that job's own work), for both precisions, and each job stops by its own
configuration."""
import numpy as np
import pytest

import oracle
import scenegen
from tests._util import pose_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2608_14266_gb300 as mm
    assert torch.cuda.is_available()
    return mm


def _job_scenes(n_jobs, seed=0):
    """Uneven jobs in the batched workload's proportions (voxels = 50 x scans,
    5-30 observations per voxel), at test sizes."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_jobs):
        n_scans = int(rng.integers(8, 40))
        p = scenegen.SceneParams(n_scans=n_scans, n_voxels=50 * n_scans, obs_min=5, obs_max=30, pts_per_obs=16,
                                 noise_sigma=0.02, rot_sigma_deg=0.5, trans_sigma=0.1, seed=5000 + k)
        s = scenegen.make_scene(p)
        pts = s.points()
        out.append((s, s.point_offsets(), pts))
    return out


def _load(mm, s, po, pts, **cfg):
    ba = mm.BundleAdjuster(**cfg)
    ba.load_points(s.n_scans, s.voxel_off, s.obs_scan, po, pts, s.pose_init)
    return ba


TOL = {"fp64": (1e-9, 1e-8, 1e-10), "mixed": (1e-6, 1e-5, 1e-6)}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_iterations_equal_alone(mm, precision):
    """A job alone (a batch of one) and in a batch of seven: identical bits."""
    prec = mm.BA_MIXED if precision == "mixed" else mm.BA_FP64
    scenes = _job_scenes(7)
    alone = []
    for s, po, pts in scenes:
        ba = _load(mm, s, po, pts, precision=prec)
        with mm.Batch() as one:
            one.add(ba)
            one.iterate(4)
            one.iterate(2)
        alone.append((ba.poses(), ba.cost(), ba.stats()["accepted"]))
        # the handle's own launches agree within the precision's tolerance
        own = _load(mm, s, po, pts, precision=prec)
        own.iterate(6)
        r, t = pose_errors(own.poses(), ba.poses())
        rt, tt, ct = TOL[precision]
        assert r < rt and t < tt
        assert own.cost() == pytest.approx(ba.cost(), rel=ct)
        own.close()
        ba.close()
    jobs = [_load(mm, s, po, pts, precision=prec) for s, po, pts in scenes]
    with mm.Batch() as b:
        for j in jobs:
            b.add(j)
        assert len(b) == len(jobs)
        b.iterate(4)
        b.iterate(2)  # a second graph (other iteration count) continues the same state
        for j, (poses, cost, acc) in zip(jobs, alone):
            np.testing.assert_array_equal(j.poses(), poses)
            assert j.cost() == cost
            assert j.stats()["accepted"] == acc
        assert b.kernel_launches() >= 3 * 6
    for j in jobs:
        j.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_of_several_job_groups_equals_alone(mm, precision):
    """More jobs than one launch parameter group holds (128): the groups run
    on separate branches of the captured graph, and every job still ends with
    the bits it reaches alone, the last, partial group included."""
    prec = mm.BA_MIXED if precision == "mixed" else mm.BA_FP64
    rng = np.random.default_rng(77)
    scenes = []
    for k in range(2 * 128 + 3):
        n_scans = int(rng.integers(3, 9))
        p = scenegen.SceneParams(n_scans=n_scans, n_voxels=20 * n_scans, obs_min=3, obs_max=8, pts_per_obs=8,
                                 noise_sigma=0.02, rot_sigma_deg=0.5, trans_sigma=0.1, seed=7100 + k)
        sc = scenegen.make_scene(p)
        scenes.append((sc, sc.point_offsets(), sc.points()))
    alone = []
    for s, po, pts in scenes:
        ba = _load(mm, s, po, pts, precision=prec)
        with mm.Batch() as one:
            one.add(ba)
            one.iterate(3)
        alone.append((ba.poses(), ba.cost()))
        ba.close()
    jobs = [_load(mm, s, po, pts, precision=prec) for s, po, pts in scenes]
    with mm.Batch() as b:
        for j in jobs:
            b.add(j)
        l0 = b.kernel_launches()
        b.iterate(3)
        # 3 iterations x 3 kernel kinds x 3 groups, plus the control and status launches
        assert b.kernel_launches() - l0 == 3 * 3 * 3 + 2
        for j, (poses, cost) in zip(jobs, alone):
            np.testing.assert_array_equal(j.poses(), poses)
            assert j.cost() == cost
    for j in jobs:
        j.close()


def test_batch_matches_oracle_for_one_job(mm):
    (s, po, pts), = _job_scenes(1, seed=3)
    cen = oracle.points_to_centred(po, pts)
    lm = oracle.LM(oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen), s.pose_init)
    for _ in range(5):
        lm.step()
    job = _load(mm, s, po, pts)
    with mm.Batch() as b:
        b.add(job)
        b.iterate(5)
    r, t = pose_errors(job.poses(), lm.poses)
    assert r < 1e-9 and t < 1e-8
    assert job.cost() == pytest.approx(lm.cost, rel=1e-10)
    job.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_solve_stops_each_job_by_its_own_rule(mm, precision):
    prec = mm.BA_MIXED if precision == "mixed" else mm.BA_FP64
    scenes = _job_scenes(5, seed=1)
    cfgs = [dict(precision=prec, rel_tol=10.0 ** -(2 + k), max_iters=40) for k in range(len(scenes))]
    alone = []
    for (s, po, pts), cfg in zip(scenes, cfgs):
        ba = _load(mm, s, po, pts, **cfg)
        with mm.Batch() as one:
            one.add(ba)
            assert one.solve(chunk=4) == 0
        alone.append((ba.stats()["iters"], ba.poses()))
        ba.close()
    jobs = [_load(mm, s, po, pts, **cfg) for (s, po, pts), cfg in zip(scenes, cfgs)]
    with mm.Batch() as b:
        for j in jobs:
            b.add(j)
        active = b.solve(chunk=4)
        assert active == 0
        assert b.done().all()
        for j, (iters, poses) in zip(jobs, alone):
            assert j.stats()["iters"] == iters
            np.testing.assert_array_equal(j.poses(), poses)
    for j in jobs:
        j.close()


def test_batch_membership_changes(mm):
    scenes = _job_scenes(4, seed=2)
    jobs = [_load(mm, s, po, pts) for s, po, pts in scenes]
    ref = []
    for s, po, pts in scenes:
        ba = _load(mm, s, po, pts)
        ba.iterate(3)
        ref.append(ba.poses())
        ba.close()
    with mm.Batch() as b:
        b.add(jobs[0])
        b.add(jobs[1])
        b.iterate(2)
        b.remove(jobs[0])
        b.add(jobs[2])
        jobs[2].iterate(2)  # a job may also run on its own between batch calls
        b.add(jobs[3])
        jobs[3].iterate(1)
        with pytest.raises(mm.BAError):
            b.add(jobs[1])  # already in
        b.iterate(1)  # jobs 1, 2 -> 3 iterations
        b.remove(jobs[3])
        b.add(jobs[0])
        b.iterate(1)  # jobs 0, 1, 2: 3, 4, 4 iterations
        jobs[3].iterate(1)
        # handle and batch launches mix here: equal within FP64 rounding
        for k in (0, 3):
            r, t = pose_errors(jobs[k].poses(), ref[k])
            assert r < 1e-12 and t < 1e-11
        with pytest.raises(mm.BAError):
            jobs[1].load_points(scenes[1][0].n_scans, scenes[1][0].voxel_off, scenes[1][0].obs_scan, scenes[1][1],
                                scenes[1][2], scenes[1][0].pose_init)
    for j in jobs:
        j.close()


def test_autotune_leaves_results_bit_identical(mm):
    """The batch tuner times its nine launch settings on the jobs' own solve
    iterations and keeps the fastest; since no candidate changes arithmetic,
    a tuned solve ends with the same bits, iteration counts and stop flags as
    an untuned one.  FP64 batches have nothing to tune."""
    scenes = _job_scenes(6, seed=4)
    cfg = dict(precision=mm.BA_MIXED, rel_tol=1e-12, max_iters=60)
    plain = [_load(mm, s, po, pts, **cfg) for s, po, pts in scenes]
    with mm.Batch() as b:
        for j in plain:
            b.add(j)
        assert b.solve(chunk=4) == 0
    ref = [(j.poses(), j.cost(), j.stats()["iters"]) for j in plain]
    tuned = [_load(mm, s, po, pts, **cfg) for s, po, pts in scenes]
    with mm.Batch() as b:
        for j in tuned:
            b.add(j)
        rep = b.autotune(iters_per_trial=1, passes=2)
        assert len(rep["candidates"]) == 9
        assert {(c["min_blocks"], c["prefetch"]) for c in rep["candidates"]} == \
            {(m, p) for m in (4, 6, 8) for p in (0, 2, 4)}
        if rep["passes"] > 0:
            ms = [c["ms_per_iter"] for c in rep["candidates"]]
            assert rep["chosen"] == int(np.argmin(ms)) and min(ms) > 0
        assert b.solve(chunk=4) == 0
    for j, (poses, cost, iters) in zip(tuned, ref):
        np.testing.assert_array_equal(j.poses(), poses)
        assert j.cost() == cost
        assert j.stats()["iters"] == iters
    for j in plain + tuned:
        j.close()
    (s, po, pts), = _job_scenes(1, seed=5)
    j = _load(mm, s, po, pts, precision=mm.BA_FP64)
    with mm.Batch() as b:
        b.add(j)
        rep = b.autotune()
        assert rep["candidates"] == [] and rep["chosen"] == -1
    j.close()


def test_autotune_cache_and_set_launch(mm, tmp_path):
    """A tuned choice is stored under the device's name; a later batch
    applies it without trials; stored or explicit settings leave the results
    bit-identical; settings outside the variants are refused."""
    import json
    scenes = _job_scenes(3, seed=6)
    cfg = dict(precision=mm.BA_MIXED, rel_tol=1e-12, max_iters=40)
    cache = str(tmp_path / "tune.json")
    runs = []
    for mode in ("tune", "cached", "explicit"):
        jobs = [_load(mm, s, po, pts, **cfg) for s, po, pts in scenes]
        with mm.Batch() as b:
            for j in jobs:
                b.add(j)
            if mode == "explicit":
                b.set_launch(4, 0)
                with pytest.raises(mm.BAError):
                    b.set_launch(5, 0)
            else:
                rep = b.autotune(iters_per_trial=1, passes=1, cache=cache)
                if mode == "cached":
                    assert rep["iterations"] == 0 and "cached" in rep
            b.solve(chunk=4)
        runs.append([(j.poses(), j.cost(), j.stats()["iters"]) for j in jobs])
        for j in jobs:
            j.close()
    table = json.load(open(cache))
    assert len(table) == 1 and set(next(iter(table.values()))) == {"min_blocks", "prefetch"}
    for other in runs[1:]:
        for (p0, c0, i0), (p1, c1, i1) in zip(runs[0], other):
            np.testing.assert_array_equal(p0, p1)
            assert c0 == c1 and i0 == i1
