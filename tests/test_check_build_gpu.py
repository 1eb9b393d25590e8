"""The -DBDM_CHECK build of the library: every index a kernel derives from
device data is range-checked, and a failed check is reported through the
device error word instead of an out-of-range access.  With compute-sanitizer
closed on this pool, this build running the small parity cases with a zero
error word is the memory-safety evidence.  The cases run in a child process
that loads the check build (the library is loaded once per process)."""
import os
import subprocess
import sys

import pytest

from paper_2301_06984_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_check_build_runs_the_parity_cases_with_no_failed_check():
    lib = B.build(variant="check")
    env = dict(os.environ, BDM_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "tests.check_build_cases"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.count("ok case_") == 8
    assert "libbdm_gb300_check.so" in r.stdout
