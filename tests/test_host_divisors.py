"""The multiply-shift division of element offsets by the row pitch and the
plane stride (Geom::div_P, div_sz, slot_of in mg_internal.h, used by the
prolongation and batched restriction kernels) agrees with integer division
on every offset of small grids and on offsets next to every multiple of the
divisor of large ones.  Host code only: compiled with nvcc, run on the CPU."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_magic_division_matches_integer_division():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "divisors_check")
        subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "host", "divisors_check.cu")],
                       check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
