"""The GPU point generator draws the same counter-based streams as the CPU
generator: same points up to the last bits of the math library."""
import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu


def test_points_device_matches_host():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    s = scenegen.make_scene(scenegen.config("tiny"))
    n_obs, npo = s.n_obs, s.params.pts_per_obs
    host = s.points()
    for o0, o1 in ((0, n_obs), (7, 7), (3, min(n_obs, 40))):
        out = torch.empty(((o1 - o0) * npo, 3), dtype=torch.float64, device="cuda")
        s.points_device(o0, o1, out)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), host[o0 * npo:o1 * npo], rtol=0, atol=1e-9)


@pytest.mark.parametrize("params", [
    dict(n_scans=37, n_voxels=1850, obs_min=5, obs_max=30, pts_per_obs=32, noise_sigma=0.02, rot_sigma_deg=0.5,
         trans_sigma=0.1, seed=9003),
    dict(n_scans=6, n_voxels=300, obs_min=5, obs_max=30, pts_per_obs=40, noise_sigma=0.0, side_min=0.5, side_max=4.0,
         degenerate_frac=0.2, perturb_scan0=True, seed=77),
])
def test_device_job_matches_host_scene(params):
    """sgd_job rebuilds the host generator's scene on the device: the same
    observation structure bit for bit, the same poses and patches up to the
    math library's last bits; its FP64 points equal the host's, and the fast
    FP32-drawn points stay within a few micrometres of them."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    p = scenegen.SceneParams(**params)
    host = scenegen.make_scene(p)
    side = torch.cuda.Stream()
    dev = scenegen.make_scene_device(p, stream=side)
    side.synchronize()
    assert dev.bad.item() == 0 and dev.n_obs == host.n_obs
    np.testing.assert_array_equal(dev.voxel_off.cpu().numpy(), host.voxel_off)
    np.testing.assert_array_equal(dev.obs_scan.cpu().numpy(), host.obs_scan)
    np.testing.assert_array_equal(dev.obs_voxel.cpu().numpy(),
                                  np.repeat(np.arange(p.n_voxels, dtype=np.int32), np.diff(host.voxel_off)))
    for name in ("pose_gt", "pose_init", "plane", "extent"):
        np.testing.assert_allclose(getattr(dev, name).cpu().numpy(), getattr(host, name), rtol=0, atol=1e-12,
                                   err_msg=name)
    npo = p.pts_per_obs
    o0, o1 = 3, host.n_obs
    ref = host.points(o0, o1)
    exact = torch.empty(((o1 - o0) * npo, 3), dtype=torch.float64, device="cuda")
    fast = torch.empty_like(exact)
    dev.points(o0, o1, exact)
    dev.points_fast(o0, o1, fast)
    torch.cuda.synchronize()
    np.testing.assert_allclose(exact.cpu().numpy(), ref, rtol=0, atol=1e-9)
    err = np.abs(fast.cpu().numpy() - ref).max()
    assert err < 2e-5, err
