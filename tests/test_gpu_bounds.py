"""The bounds-checked build: every index the kernels compute is checked against
its array in a separate library (-DRLT2_BOUNDS_CHECK), which counts an
out-of-range index and uses 0 instead of dereferencing it.  A child process
runs every entry point on small problems with that library (tests/bounds_cases.py):
results must match the oracle and no index may have been out of range.  The
class-owned moves are race-free by construction (each z and y has one owner);
this covers the index arithmetic."""
import json
import os
import subprocess
import sys

import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_clean():
    from paper_1710_03732_gb300 import build
    lib = build.build(checked=True)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), lib], capture_output=True, text=True,
                       timeout=900)
    assert r.stdout.strip(), r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    failed = [name for name, ok in out["checks"] if not ok]
    assert not failed and r.returncode == 0, (failed, r.stderr[-2000:])
    assert out["violations"] == 0


def test_normal_build_reports_no_counter():
    from paper_1710_03732_gb300 import build, rlt2
    build.build()
    assert rlt2.rlt2_debug_bounds_violations() == -1
