"""The mixed form's FP64 -> FP32 narrowing and FP32 -> FP64 widening
(integer-only, cycle_device.cuh) against CUDA's own conversions on the GPU:
round toward zero (__double2float_rz) bit for bit in the normal range and
at overflow, the documented flush below 2^-126, infinities kept and NaN
never produced from a finite value (tests/host/convert_check.cu)."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

pytestmark = pytest.mark.gpu


def test_conversions_match_cuda_round_toward_zero():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    assert os.path.exists(nvcc), "nvcc not found"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "convert_check")
        subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                        os.path.join(HERE, "host", "convert_check.cu")], check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
