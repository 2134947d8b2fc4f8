"""The cell numbering (tiles of T x T x T cells, T = 1, 2 or 4 by build) is
a bijection with the documented order and an exact inverse: a host build of
the library's own helpers (tests/cellorder_check.cu) for each T."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("tile", [1, 2, 4])
def test_cell_numbering(tmp_path, tile):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / f"cellorder_check{tile}")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                        f"-DMD_CELL_TILE={tile}", "-o", exe, os.path.join(HERE, "cellorder_check.cu")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok:")
