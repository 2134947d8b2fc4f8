"""The double-word building blocks of the MD_DW kernels (dw_arith.cuh) and
the position split (dw_split), built for the host from the same source with
floating-point contraction off, against exact and long-double references
(tests/dw_arith_check.cu): the error-free transformations are exact, the
double-word product, sum, r^2, reciprocal and reciprocal square root stay
within their stated bounds, the split keeps the high parts on the grid with
exact differences, and the LJ force factor chain is good to 4e-13."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_double_word_building_blocks(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "dw_arith_check")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off",
                        "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                        os.path.join(HERE, "dw_arith_check.cu")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe, "200000"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok:")
