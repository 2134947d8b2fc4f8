"""md_study_force_variant: the force-kernel variants that the design notes
compare with the library's kernel compute the same forces.  SoA and AoSoA
gathers, and gathers through the texture path, run the library's arithmetic
in its order (bitwise equal forces); the
shared-memory tile variant rounds differently (tile frame) and is held to
the mixed path's tolerance against the oracle; staged by TMA bulk copies
instead of loads it gives the same bits."""
import numpy as np
import pytest

from paper_2009_07400_gb300 import inputs

pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_07400_gb300 import build
    build.build()
    from paper_2009_07400_gb300 import md as m
    m.load()
    return m


def rms_rel(F, Fr):
    return np.sqrt(np.sum((F - Fr) ** 2) / np.sum(Fr ** 2))


@pytest.mark.parametrize("case", ["liquid", "small_box", "odd_cells"])
def test_study_variants_agree(md, orc, case):
    if case == "liquid":
        s = inputs.fcc_system(7, jitter=0.05, seed=3)
        x, v, _ = orc.vv_run(s.pos, s.vel, s.box, 40)
        s = inputs.System(x, v, s.box, 3)
    elif case == "small_box":                      # 2 cells per edge: every cell staged twice
        s = inputs.replica_system(270, 0.8, 1.0, seed=4)
    else:                                          # 7 cells per edge: tiles stick out of the box
        s = inputs.fcc_system(12, jitter=0.05, seed=5)
    nc = np.floor(np.asarray(s.box) / (RC + SKIN)).astype(int)
    assert {"small_box": 2, "odd_cells": 7}.get(case, nc[0]) == nc[0]
    xw = orc.wrap(s.pos, s.box)
    Fr = orc.forces_list(xw, s.box, orc.neighbors_cells(xw, s.box, RC + SKIN))
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, threads_per_atom=1) as ctx:
        F_lib = ctx.forces()
        us0, F0 = ctx.study_force_variant(0, 2, forces=True)
        assert us0 > 0 and np.array_equal(F0, F_lib)
        for v in (1, 2, 5, 6):                   # layouts, texture-path gathers
            us, F = ctx.study_force_variant(v, 2, forces=True)
            assert us > 0 and np.array_equal(F, F0)
        _, F3 = ctx.study_force_variant(3, 2, forces=True)
        assert rms_rel(F3, Fr) <= 1e-5
        _, F4 = ctx.study_force_variant(4, 2, forces=True)      # staged by TMA bulk copies
        assert np.array_equal(F4, F3)
        assert np.array_equal(ctx.forces(), F_lib)        # the context's state is untouched


def test_study_rejects_other_contexts(md, orc):
    s = inputs.fcc_system(5, jitter=0.05, seed=6)
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_FP64) as ctx:
        with pytest.raises(md.MDError) as e:
            ctx.study_force_variant(1, 1)
        assert e.value.code == md.MD_ERR_STATE
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, half_list=True) as ctx:
        with pytest.raises(md.MDError) as e:
            ctx.study_force_variant(0, 1)
        assert e.value.code == md.MD_ERR_STATE
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED) as ctx:
        with pytest.raises(md.MDError) as e:
            ctx.study_force_variant(7, 1)
        assert e.value.code == md.MD_ERR_INVAL
