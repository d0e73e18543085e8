"""Run by test_gpu_checked.py in a process that loads the checked library
(MMBA_CHECKED=1, kernels with index checks): solves of the tiny scene in both
precisions, a batch of uneven jobs and a voxelisation, each compared with the
oracle.  A kernel index out of range would make a call raise (BA_ERR_STATE)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import paper_2608_14266_gb300 as mm  # noqa: E402
import scenegen  # noqa: E402
from tests._util import pose_errors  # noqa: E402

assert mm._lib.LIB_PATH.endswith("libmmba_checked.so"), mm._lib.LIB_PATH
s = scenegen.make_scene(scenegen.config("tiny"))
pts, po = s.points(), s.point_offsets()
cen = oracle.points_to_centred(po, pts)
lm = oracle.LM(oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen), s.pose_init)
for _ in range(5):
    lm.step()
for prec, rtol in ((mm.BA_FP64, 1e-10), (mm.BA_MIXED, 1e-6)):
    with mm.BundleAdjuster(precision=prec) as ba, mm.BundleAdjuster() as ev:
        ba.load_points(s.n_scans, s.voxel_off, s.obs_scan, po, pts, s.pose_init)
        ba.iterate(5)
        ev.load_points(s.n_scans, s.voxel_off, s.obs_scan, po, pts, ba.poses())
        c_ref, _ = oracle.voxel_pass(oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan, cen), ba.poses())
        assert abs(ba.cost() - c_ref) <= rtol * c_ref, (prec, ba.cost(), c_ref)
        if prec == mm.BA_FP64:
            r, t = pose_errors(ba.poses(), lm.poses)
            assert r < 1e-9 and t < 1e-8, (r, t)
jobs = []
for k in range(3):
    p = scenegen.SceneParams(n_scans=8 + 5 * k, n_voxels=400 + 100 * k, obs_min=3, obs_max=12, pts_per_obs=12,
                             noise_sigma=0.02, rot_sigma_deg=0.5, trans_sigma=0.1, seed=9300 + k)
    sk = scenegen.make_scene(p)
    ba = mm.BundleAdjuster(precision=mm.BA_MIXED)
    ba.load_points(sk.n_scans, sk.voxel_off, sk.obs_scan, sk.point_offsets(), sk.points(), sk.pose_init)
    jobs.append(ba)
with mm.Batch() as b:
    for j in jobs:
        b.add(j)
    b.iterate(4)
for j in jobs:
    j.close()
order = np.argsort(s.obs_scan, kind="stable")
P = pts.reshape(s.n_obs, s.params.pts_per_obs, 3)[order].reshape(-1, 3)
spo = np.concatenate([[0], np.cumsum(np.bincount(s.obs_scan, minlength=s.n_scans) * s.params.pts_per_obs)])
got = mm.voxelize(spo.astype(np.int64), P, s.pose_gt, 1.0, levels=3)
ref = oracle.voxelize(spo.astype(np.int64), P, s.pose_gt, 1.0, levels=3)
assert np.array_equal(got["voxel_off"], ref["voxel_off"]) and np.array_equal(got["obs_scan"], ref["obs_scan"])
print("ok")
