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
