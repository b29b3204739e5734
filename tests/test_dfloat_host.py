"""The FP64 <-> double-float conversions of the double-float transform passes
(csrc/dfloat.cuh: hi = the first 24 bits of x, lo = the next bits rounded,
from the bit pattern on the integer pipe; back to FP64 with one addition),
compiled for the host and checked against exact arithmetic on random values
over the whole FP32 exponent range, zeros and both signs (no GPU needed)."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_conversions_exact_to_2pow_minus_47(tmp_path):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "dfloat_conversions")
    src = os.path.join(HERE, "host", "dfloat_conversions.cu")
    res = subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, src], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    worst = float(run.stdout.split()[1])
    assert worst <= 2.0 ** -47
