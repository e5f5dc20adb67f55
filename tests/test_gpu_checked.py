"""The checked build of the library (-DSUPRA_CHECKED): the kernels check their index and
alignment invariants (every in-aperture sample pair inside its element's staged window,
tensor-copy and bulk-copy alignment, staged scan-conversion indices) and report a failure
as SUPRA_EINTERNAL through the device status word.  The parity suite runs against it in a
child process; each module of that suite ends by asserting a clean status word."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_passes_on_the_checked_build():
    from paper_1711_06127_b300 import build

    lib = build.build(checked=True)
    env = dict(os.environ, SUPRA_LIBRARY=lib)
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_gpu_parity.py"),
                          os.path.join(ROOT, "tests", "test_gpu_faults.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
