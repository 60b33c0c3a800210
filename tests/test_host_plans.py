"""Host-side logic of the CUDA path that needs no GPU: the work plan of the
group-cooperative humanoid kernel, built by the same host code the library
runs, checked for complete and exclusive coverage (tests/host/)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not available")


def test_group_plan_covers_every_task_once():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "group_plan_check")
        src = os.path.join(ROOT, "tests", "host", "group_plan_check.cu")
        r = subprocess.run([_nvcc(), "-std=c++17", "--expt-relaxed-constexpr", "-O1", "-I",
                            os.path.join(ROOT, "include"), src, "-o", exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-3000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stdout[-3000:]
        assert "humanoid36: 0 problems" in r.stdout and "humanoid36_hull: 0 problems" in r.stdout
