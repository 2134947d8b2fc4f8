"""md_energy_sums_static: FP64 energy totals without any device allocation.

Some callers cannot allocate device memory where they need these totals: an
external engine that owns the whole GPU through its own memory pool, a
deployment with a fixed device-memory budget, or a loop that must not call
cudaMalloc because it can synchronise the device.  The entry point takes
their per-atom inputs and an output slot and keeps its only scratch in a
fixed array inside the library.  Here it is called through the C ABI twice
in a row (a three-chunk system, then a one-chunk system, so a stale partial
of the first call would show) and checked against md_energy on the same
states, with the FP64 energy tolerances of the other parity tests.
"""
import numpy as np
import pytest

from paper_2009_07400_gb300 import inputs

RC, SKIN = 2.5, 0.3


@pytest.fixture(scope="module")
def md():
    from paper_2009_07400_gb300 import build
    build.build()
    from paper_2009_07400_gb300 import md as m
    m.load()
    return m


def test_rejects_sizes_beyond_the_fixed_scratch(md):
    """n above the stated maximum fails before any device work."""
    with pytest.raises(md.MDError) as e:
        md.energy_sums_static(33554432 + 1, 1, 1, 1, 1.0, 1)
    assert e.value.code == -1
    assert "exceeds the maximum of 33554432" in str(e.value)


@pytest.mark.gpu
def test_static_sums_match_md_energy(md, orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    s_big = inputs.replica_system(9000, 0.84, 1.2, seed=17)            # 3 chunks of 4096
    s_small = inputs.fcc_system(7, jitter=0.05, seed=3)                # 1 chunk
    x, v, _ = orc.vv_run(s_small.pos, s_small.vel, s_small.box, 30)
    s_small = inputs.System(x, v, s_small.box, 3)
    stream = torch.cuda.current_stream()
    for s in (s_big, s_small):
        with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_FP64) as ctx:
            pe, ke, w = (q[0] for q in ctx.energy())
        xw = orc.wrap(s.pos, s.box)
        rows = orc.neighbors_cells(xw, s.box, RC + SKIN, half=True)
        pe_a, w_a = orc.energy_atoms(xw, s.box, rows, half=True)
        d_pe = torch.tensor(pe_a, dtype=torch.float64, device="cuda")
        d_w = torch.tensor(w_a, dtype=torch.float64, device="cuda")
        d_v = torch.tensor(np.ascontiguousarray(s.vel), dtype=torch.float64, device="cuda")
        out = torch.full((3,), np.nan, dtype=torch.float64, device="cuda")
        md.energy_sums_static(s.n, d_pe.data_ptr(), d_w.data_ptr(), d_v.data_ptr(), 1.0,
                              out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(pe, rel=1e-12)
        assert got[1] == pytest.approx(ke, rel=1e-13)
        assert got[2] == pytest.approx(w, rel=1e-11)
