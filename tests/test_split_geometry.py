"""CPU checks of host-side index and factor logic built from the CUDA sources (no GPU needed):
tests/split_geometry_check.cu includes the factored solver's source and checks every sub-line
it builds for lines of 4300 to 16384 cells, halos 1 to 16, FP32 and FP64;
tests/prologue_factor_check.cu checks the prologue's precomputed Thomas factors against a
dense elimination of the App. A matrices."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _build_and_run(name):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = os.path.join(HERE, "_build")  # git-ignored
    os.makedirs(out, exist_ok=True)
    exe = os.path.join(out, name)
    cmd = [nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I" + os.path.join(ROOT, "include"),
           "-o", exe, os.path.join(HERE, name + ".cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "bad 0" in r.stdout, r.stdout[-2000:]


def test_split_line_geometry_host_check():
    _build_and_run("split_geometry_check")


def test_prologue_thomas_factors_host_check():
    _build_and_run("prologue_factor_check")
