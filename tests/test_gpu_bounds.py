"""The bounds-checking build (-DFDTD_CHECK_BOUNDS, the stand-in for a
memory checker): every shared-memory access and output store of the TMA
tile pipelines is tested against its allocation; the small, ragged cases of
tests/bounds_cases.py must count none outside."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_counts_no_out_of_bounds_access():
    sys.path.insert(0, os.path.join(ROOT, "paper_0904_0939_gb300"))
    build = subprocess.run([sys.executable, os.path.join(ROOT, "paper_0904_0939_gb300", "_build.py"), "--checked"],
                           capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-2000:]
    lib = build.stdout.strip().splitlines()[-1]
    assert lib.endswith("libfdtd_checked.so") and os.path.exists(lib)
    env = dict(os.environ, FDTD_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_cases.py")], capture_output=True,
                       text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["cases"] >= 100
    assert out["violations"] == 0
