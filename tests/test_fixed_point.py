"""The averaging arithmetic of the half-pass kernels, checked on the CPU.

The deferred mean of Alg. 1 ("MMA") is formed from a 64-bit fixed-point sum of the masses
the slots remove. ``tests/native/fixed_point_check.cu`` compiles the kernels' own helpers
(``csrc/device_util.cuh``) for the host and compares them with exact integer and
extended-precision arithmetic: the integer value of an integer-valued float, the rounding of
a mass to the grid (ties to even), the exact split of a sum into a double-float, the mean
for every degree, and sums of rounded masses.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fixed_point_helpers_match_exact_arithmetic(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "fixed_point_check")
    src = os.path.join(HERE, "native", "fixed_point_check.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-gencode",
                        "arch=compute_103a,code=sm_103a", "-o", exe, src], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
