"""The kernels split cell indices with a multiply-shift division by invariant integers;
its host copy (the same header code) is checked against true division by brute force."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fast_division_matches_integer_division(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "fastdiv_check"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", str(exe), os.path.join(HERE, "native", "fastdiv_check.cu")],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
