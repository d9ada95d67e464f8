"""The GPU parity suite once more on the checked build (-DBS_CHECK=1): every
kernel tests each index it reads from memory, and the binding collects the
device-side check words after every library call (bs_check_device), raising
on any recorded failure.  On the suite's valid inputs no check may fire, and
every test must still pass with the checks in the kernels.  The inputs are
the suite's own: nothing out of range is given to the GPU."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_on_the_checked_build():
    from paper_2009_10917_gb300 import build
    path = build.build(check=True)
    env = dict(os.environ, BS_CHECK="1")
    probe = ("from paper_2009_10917_gb300 import bs; L = bs.lib(); "
             "assert bs.checked() and L.bs_check_enabled() == 1; print(bs.library_path())")
    r = subprocess.run([sys.executable, "-c", probe], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == path
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-q", "-x",
                        "-p", "no:cacheprovider",
                        "--ignore", os.path.join("tests", "test_zz_checked_build.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=2400)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-30:])
    assert r.returncode == 0, tail
    assert " passed" in tail and "device check" not in tail
