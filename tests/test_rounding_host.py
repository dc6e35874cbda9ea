"""Host check of the hash behind the 16-bit stochastic rounding's random bits
(csrc/lbm_round.cuh): built with nvcc for the CPU and run here; see
tests/host/sr_check.cu (hash invertible, hashed starts uniform).  The
conversions are device instructions: tests/test_rounding_gpu.py."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_rounding_hash_is_a_uniform_bijection(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "sr_check")
    src = os.path.join(ROOT, "tests", "host", "sr_check.cu")
    inc = os.path.join(ROOT, "paper_2011_15073_gb300", "csrc")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", inc, src, "-o", exe], check=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:]
    assert r.stdout.startswith("OK")
