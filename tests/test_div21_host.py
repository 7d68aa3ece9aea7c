"""The pivot reciprocal's 2-by-1 limb division (div21_preinv with its
precomputed reciprocal, Moller and Granlund 2011, Alg. 4) compiled for the CPU
from the kernels' own header and checked against exact division on about six
million dividend and divisor pairs (tests/host/div21_check.cu).  Needs nvcc
for the host compile; no GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_div21_preinv_equals_exact_division(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = tmp_path / "div21_check"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-o", str(exe), os.path.join(HERE, "host", "div21_check.cu")])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
