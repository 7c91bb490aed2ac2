"""The checked build (MSK_CHECKED: device-side index checks that record the
site of a failed check instead of touching memory) runs the CountSketch
family, the sliced FP64 Gaussian stage, a refined solve and a batch in a child
process, each result against the oracle, and no check fails."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_clean():
    from paper_2508_14209_gb300 import build

    lib = build.build(checked=True)
    env = dict(os.environ, MSK_LIB=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_checked_run.py")], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=1200)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-3000:]
    assert "all cases passed" in out.stdout
