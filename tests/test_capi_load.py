"""The C-ABI library builds, loads and exports every symbol include/md.h
declares; host-side argument validation works without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_07400_gb300 import build, md
    build.build()
    return md.load()


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(md_[a-z_0-9]+)\s*\(", text))
    return names


def test_exports_match_header(lib):
    from paper_2009_07400_gb300 import md
    declared = declared_symbols()
    assert declared == set(md.ABI_SYMBOLS)
    for name in declared:
        assert hasattr(lib, name), name


def test_library_is_cuda_native(lib):
    """The package carries no CPU compute path: the binding only marshals."""
    src = open(os.path.join(ROOT, "paper_2009_07400_gb300", "md.py")).read()
    assert "import oracle" not in src and "from oracle" not in src


def test_missing_library_fails_loudly(tmp_path):
    from paper_2009_07400_gb300 import md
    with pytest.raises(RuntimeError):
        md._lib_saved = md._lib
        try:
            md._lib = None
            md.load(str(tmp_path / "nope.so"))
        finally:
            md._lib = md._lib_saved


def _create(lib, box, params, n=4, pos=None):
    from paper_2009_07400_gb300 import md
    pos = np.zeros((n, 3)) if pos is None else pos
    vel = np.zeros((n, 3))
    b = md.md_box(*box)
    h = ctypes.c_void_p()
    rc = lib.md_create(ctypes.byref(b), ctypes.byref(params), n,
                       pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       vel.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, ctypes.byref(h))
    return rc, h


def test_host_validation_without_gpu(lib):
    from paper_2009_07400_gb300 import md
    p = md.make_params()
    rc, h = _create(lib, (5.0, 20.0, 20.0), p)            # 5.0 < 2 (rc + skin)
    assert rc == -2 and not h.value
    assert b"2 (rc + skin)" in lib.md_last_error(None)
    bad = md.make_params(dt=-1.0)
    rc, _ = _create(lib, (20.0, 20.0, 20.0), bad)
    assert rc == -1
    bad = md.make_params(threads_per_atom=3)
    rc, _ = _create(lib, (20.0, 20.0, 20.0), bad)
    assert rc == -1
    pos = np.zeros((4, 3))
    pos[2, 1] = np.nan
    rc, _ = _create(lib, (20.0, 20.0, 20.0), p, pos=pos)
    assert rc == -7
    # precisions: MD_FP64, MD_MIXED, MD_DW; the double-word path runs full
    # per-atom lists only, the group lists the mixed path only
    rc, _ = _create(lib, (20.0, 20.0, 20.0), md.make_params(precision=3))
    assert rc == -1
    for lt in (md.MD_LIST_HALF, md.MD_LIST_GROUP2, md.MD_LIST_GROUP4):
        rc, _ = _create(lib, (20.0, 20.0, 20.0), md.make_params(precision=md.MD_DW, list_type=lt))
        assert rc == -1
    assert b"full per-atom lists" in lib.md_last_error(None) or b"mixed path" in lib.md_last_error(None)


def _create_batch(lib, boxes, counts, params, pos=None):
    from paper_2009_07400_gb300 import md
    n_pos = max(1, min(int(sum(counts)), 8))
    pos = np.zeros((n_pos, 3)) if pos is None else pos
    barr = (md.md_box * len(boxes))(*[md.md_box(*b) for b in boxes])
    cnt = np.asarray(counts, np.int64)
    h = ctypes.c_void_p()
    rc = lib.md_create_batch(len(boxes), barr, ctypes.byref(params),
                             cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None,
                             ctypes.byref(h))
    return rc, h


def test_size_limits_rejected_before_device_work(lib):
    """Limits are checked on the host before any array is read or any
    device memory is touched (the position array here is deliberately tiny)."""
    from paper_2009_07400_gb300 import md
    p = md.make_params()
    rc, h = _create_batch(lib, [(20.0, 20.0, 20.0)], [0], p)
    assert rc == -1 and not h.value                            # empty replica
    rc, h = _create_batch(lib, [(20.0, 20.0, 20.0)], [1 << 26], p)
    assert rc == -1 and b"67,108,863" in lib.md_last_error(None)
    rc, h = _create_batch(lib, [(1024 * 2.8 + 1.0, 20.0, 20.0)], [4], p)
    assert rc == -1 and b"1023 cells" in lib.md_last_error(None)
    rc, h = _create_batch(lib, [(20.0, 20.0, 20.0), (5.0, 20.0, 20.0)], [2, 2], p)
    assert rc == -2                                            # second box too small


def test_device_entry_points_reject_host_memory(lib):
    """md_create_device checks that pos/vel are device memory before any
    device work (here there is no device at all, or the arrays are host)."""
    from paper_2009_07400_gb300 import md
    p = md.make_params()
    pos = np.zeros((4, 3))
    b = md.md_box(20.0, 20.0, 20.0)
    h = ctypes.c_void_p()
    rc = lib.md_create_device(ctypes.byref(b), ctypes.byref(p), 4,
                              ctypes.c_void_p(pos.ctypes.data), ctypes.c_void_p(pos.ctypes.data),
                              None, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert b"not device pointers" in lib.md_last_error(None)
