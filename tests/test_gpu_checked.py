"""The checked library variant (kernel index checks compiled in, a stand-in
for a memory sanitizer, which is closed on this machine) runs the tiny scene's
solves, a batch and a voxelisation without an index out of range, and agrees
with the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_clean():
    import torch
    assert torch.cuda.is_available()
    from paper_2608_14266_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, MMBA_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert r.stdout.strip().endswith("ok")
