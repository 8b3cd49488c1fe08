"""The checked build (QLC_CHECKED: every index the kernels compute from data
is range-checked; a failure records its site and sets QLC_ERR_CHECK, never a
trap) runs small parity cases, corrupt containers and batches included, with
no check failing and every byte equal to the oracle's.  The checks stand in
for a memory checker (compute-sanitizer is not available on the test GPUs)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_small_parity_cases():
    from paper_2602_17849_gb300 import _build
    lib = _build.build(checked=True)
    env = dict(os.environ, QLC_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_checked_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no index check failed" in r.stdout


def test_normal_build_reports_no_checks():
    """The normal library is not the checked one: its check hook answers
    0xFFFFFFFF."""
    import ctypes

    from paper_2602_17849_gb300 import qlc
    if os.environ.get("QLC_LIBRARY"):
        pytest.skip("QLC_LIBRARY names another build")
    qlc.lib.qlc_test_check_take.restype = ctypes.c_uint32
    assert qlc.lib.qlc_test_check_take() == 0xFFFFFFFF
