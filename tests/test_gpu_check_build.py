"""The bounds-check build (SKEI_CHECK = 1; no memory checker is open on this
GPU pool): small cases of every instrumented kernel family run against
libskei_check.so in a process of their own, with NaN guard bands around
every output; no range check may fire, no guard may change, and every
result must match the FP64 oracle (tests/_check_cases.py)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_small_cases_under_range_checks():
    from paper_2411_05771_gb300 import build
    lib = build.build(check=True)
    env = dict(os.environ, SKEI_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_check_cases.py")],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "CHECK_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_normal_build_reports_no_checks():
    from paper_2411_05771_gb300 import skei as S
    assert not S.check_build()
    assert S.check_status() == 0
