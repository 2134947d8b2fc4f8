"""The FP64/FP32 conversions and compares that the kernels perform on IEEE
bit patterns (to keep them off GB300's narrow FP64 pipe) give the hardware
conversions' results bit for bit: a host build of the library's own helpers
(tests/bitconv_check.cu) checks every float and millions of doubles, exact
rounding ties and edge cases included."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bit_pattern_conversions_match_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "bitconv_check")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-o", exe, os.path.join(HERE, "bitconv_check.cu")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe, "2000000"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok:")
