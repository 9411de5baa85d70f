"""The checked build (-DMD_CHECKED, device-side bounds checks that latch
MD_ERR_BOUNDS instead of trapping): the cases of tests/checked_cases.py run in
a child process that loads libmd_gb300_checked.so (MD_GB300_CHECKED=1).  The
checks take the place of a memory checker, which this library does not rely
on."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_cases(report):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, MD_GB300_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", os.path.join("tests", "checked_cases.py"), "-q", "-x",
           "-p", "no:cacheprovider"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    tail = "\n".join((r.stdout + r.stderr).strip().splitlines()[-30:])
    assert r.returncode == 0, tail
    report("checked build: " + tail.splitlines()[-1])
