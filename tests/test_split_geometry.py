"""CPU check of the split-line geometry of the factored solver (no GPU needed): compiles
tests/split_geometry_check.cu, which includes the solver's source and checks every sub-line
it builds for lines of 4300 to 16384 cells, halos 1 to 16, FP32 and FP64, then runs it."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_split_line_geometry_host_check():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = os.path.join(HERE, "_build")  # git-ignored
    os.makedirs(out, exist_ok=True)
    exe = os.path.join(out, "split_geometry_check")
    cmd = [nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I" + os.path.join(ROOT, "include"),
           "-o", exe, os.path.join(HERE, "split_geometry_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "bad 0" in r.stdout, r.stdout[-2000:]
