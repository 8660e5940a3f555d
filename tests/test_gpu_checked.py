"""The bounds-checked build (-DLC_CHECKED): every index a kernel takes from
data (CSR columns, the local domain's index maps, the batched systems'
compacted columns) is tested against its range, and a failure is recorded in
a device status word instead of being accessed.  It stands in for a memory
checker: the whole GPU suite runs once more on that build, and each test must
end with no recorded failure (the autouse fixture in conftest.py).  A
positive control shows that a failing index is recorded, located and cleared.
"""
import os
import subprocess
import sys

import pytest

from paper_2001_01158_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CONTROL = r"""
import torch, paper_2001_01158_gb300 as lcg
assert lcg.checked_status() == (0, "")
lcg.checked_selftest()
torch.cuda.synchronize()
n, where = lcg.checked_status()
assert n == 1 and where.startswith("lc_api.cu:"), (n, where)
assert lcg.checked_status() == (0, "")   # collected records are cleared
print("control ok", where)
"""


def _env():
    env = dict(os.environ)
    env["LC_CHECKED"] = "1"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    return env


@pytest.fixture(scope="module")
def checked_lib():
    return build_library(checked=True)


@pytest.mark.gpu
def test_checked_build_records_a_failing_index(checked_lib):
    p = subprocess.run([sys.executable, "-c", CONTROL], cwd=ROOT, env=_env(), capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "control ok" in p.stdout


@pytest.mark.gpu
def test_gpu_suite_is_clean_under_the_checked_build(checked_lib):
    cmd = [sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider",
           "--ignore", os.path.join("tests", "test_gpu_checked.py")]
    p = subprocess.run(cmd, cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=1500)
    tail = "\n".join((p.stdout + p.stderr).splitlines()[-30:])
    assert p.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail, tail
