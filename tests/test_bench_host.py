"""Host-side logic of bench.py (no GPU): the algorithmic-bytes figure of the
roofline, the pinned tuner choice of profiling commands, the check that ties
the committed ncu traffic to the current force-kernel source, and the JSON
line of the oracle (reference) arm."""
import hashlib
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_per_atom():
    # full list, fused step: 4 k + 4 (row length) + 16 + 16 (p32 in/out)
    # + 2 x 24 (x in/out) + 2 x 24 (v in/out)
    assert bench.algorithmic_bytes_per_atom(75.0, 0) == 4 * 75 + 4 + 32 + 96
    # half list, force only: entries, row length, p32 in, force out
    assert bench.algorithmic_bytes_per_atom(37.5, 1) == 4 * 37.5 + 4 + 32
    # group list of 4, fused step: entries and their member bytes per atom,
    # row length, group table entry and pair mask per group (0.27 per atom)
    assert bench.algorithmic_bytes_per_atom(35.0, 4, 0.27) == 5 * 35 + 10 * 0.27 + 32 + 96


def test_parse_tuned():
    assert bench.parse_tuned(None) is None
    assert bench.parse_tuned("") is None
    mixed, fp64, dw = bench.parse_tuned("1,0,2,1")
    assert mixed == {"threads_per_atom": 1, "list_type": 0}
    assert fp64 == {"threads_per_atom": 2, "list_type": 1}
    assert dw is None
    assert bench.parse_tuned("1,4,2,0")[0] == {"threads_per_atom": 1, "list_type": 4}
    assert bench.parse_tuned("1,0,2,0,4")[2] == {"threads_per_atom": 4, "list_type": 0}
    for bad in ("3,0,1,0", "1,0,1", "1,0,16,0", "1,3,1,0", "1,0,1,4", "1,0,1,0,3",
                "1,0,1,0,1,1"):
        with pytest.raises(SystemExit):
            bench.parse_tuned(bad)


def test_ncu_traffic_follows_the_kernel_source():
    """The committed DRAM traffic is reported only while its recorded hash
    matches the force kernel's source; a changed kernel reports null."""
    current = hashlib.sha256(open(bench.FORCE_SRC, "rb").read()).hexdigest()
    for lt, path in bench.PROFILE_MD.items():
        t = bench.ncu_traffic(lt)
        if not os.path.exists(path):
            assert t is None
            continue
        text = open(path).read()
        recorded = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text).group(1)
        if recorded == current:
            assert t is not None and 1e8 < t < 6e8     # 250-450 B per atom at 1M atoms
        else:
            assert t is None


def test_reference_arm_line():
    """--impl reference times the oracle on a bounded sample and prints one
    JSON line with the native arm's metric and unit."""
    import time
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    wall = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "atom-timesteps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the timed region (ms_per_step x steps) lies inside the process's run,
    # and the value is the atoms x time steps of that region over its length
    assert d["ms_per_step"] * d["steps"] / 1e3 < wall
    ts = d["config"]["timesteps_per_step"]
    assert d["value"] == pytest.approx(d["config"]["atoms"] * ts * d["steps"]
                                       / (d["ms_per_step"] * d["steps"] / 1e3), rel=1e-9)
