"""FP64 CPU oracle for short-range LJ 12-6 MD — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never links, loads or
calls it, and it shares no code with the CUDA library.  The arithmetic lives
in plain C (``md_oracle.c``, ``md_oracle_adjoint.c``), compiled with
``-ffp-contract=off`` so every FP64 operation is rounded as written; this
module only marshals numpy arrays.

Paper: tinyMD (Machado et al., arXiv 2009.07400).  Each C function cites the
section / equation it follows (Sec. 3.2 Eq. 1-2 and Fig. 1; Sec. 4.2 potential
kernel; Sec. 6 workload settings).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["md_oracle.c", "md_oracle_adjoint.c"]
_LIB_PATH = os.path.join(_HERE, "_liboracle_md.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_liboracle_md.so`` (gcc, FP64, no FMA
    contraction, OpenMP when available).  Returns the library path."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", tmp] + srcs + ["-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("epsilon", ctypes.c_double), ("sigma", ctypes.c_double),
                ("mass", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("skin", ctypes.c_double), ("dt", ctypes.c_double),
                ("rebuild_every", ctypes.c_int32), ("half", ctypes.c_int32),
                ("potential", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("k_spring", ctypes.c_double), ("gamma", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            sig = {
                "orc_num_threads": (ctypes.c_int, []),
                "orc_set_num_threads": (None, [ctypes.c_int]),
                "orc_cell_grid": (ctypes.c_int, [_D, ctypes.c_double, _I32, _D]),
                "orc_wrap": (None, [ctypes.c_int64, _D, _D]),
                "orc_bin": (None, [ctypes.c_int64, _D, _I32, _D, _I32, _I32, _I32]),
                "orc_neighbors_brute": (ctypes.c_int32, [ctypes.c_int64, _D, _D, ctypes.c_double,
                                                         ctypes.c_int32, ctypes.c_int32, _I32, _I32]),
                "orc_neighbors_cells": (ctypes.c_int32, [ctypes.c_int64, _D, _D, _I32, _I32, _I32,
                                                         _I32, ctypes.c_double, ctypes.c_int32,
                                                         ctypes.c_int32, _I32, _I32]),
                "orc_forces_list": (None, [ctypes.c_int64, _D, _D, ctypes.c_int32, _I32, _I32, P, _D]),
                "orc_forces_brute": (None, [ctypes.c_int64, _D, _D, P, _D]),
                "orc_forces_sample": (None, [ctypes.c_int64, _D, _D, _I32, _I32, _I32, _I32, P,
                                             ctypes.c_int64, _I64, _D]),
                "orc_energy_list": (None, [ctypes.c_int64, _D, _D, ctypes.c_int32, _I32, _I32, P,
                                           _D, _D, _D]),
                "orc_kinetic": (ctypes.c_double, [ctypes.c_int64, _D, ctypes.c_double]),
                "orc_neighbors_sample": (ctypes.c_int32, [ctypes.c_int64, _D, _D, _I32, _I32, _I32,
                                                          _I32, ctypes.c_double, ctypes.c_int64,
                                                          _I64, ctypes.c_int32, _I32, _I32]),
                "orc_thermo": (None, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int64, ctypes.c_double, _D]),
                "orc_forces_sd_list": (None, [ctypes.c_int64, _D, _D, _D, ctypes.c_int32, _I32,
                                              _I32, P, _D]),
                "orc_forces_sd_brute": (None, [ctypes.c_int64, _D, _D, _D, P, _D]),
                "orc_energy_sd_list": (None, [ctypes.c_int64, _D, _D, _D, ctypes.c_int32, _I32,
                                              _I32, P, _D, _D, _D]),
                "orc_energy_atoms": (None, [ctypes.c_int64, _D, _D, ctypes.c_int32, _I32, _I32, P,
                                            _D, _D]),
                "orc_vv_run": (ctypes.c_int, [ctypes.c_int64, _D, P, _D, _D, _D, ctypes.c_int64,
                                              ctypes.c_int64, _D]),
                "orc_jvp": (ctypes.c_int, [ctypes.c_int64, _D, P, _D, _D, _D]),
                "orc_traj_loss": (ctypes.c_int, [ctypes.c_int64, _D, P, _D, _D, ctypes.c_int64,
                                                 ctypes.c_int64, _D]),
                "orc_traj_loss_ex": (ctypes.c_int, [ctypes.c_int64, _D, P, _D, _D, ctypes.c_int64,
                                                    ctypes.c_int64, _D, ctypes.c_int,
                                                    ctypes.POINTER(ctypes.c_void_p)]),
                "orc_trace_free": (None, [ctypes.c_void_p]),
                "orc_adjoint": (ctypes.c_int, [ctypes.c_int64, _D, P, _D, _D, ctypes.c_int64,
                                               ctypes.c_int64, _D, _D, _D, _D, _D]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I32)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _box(L):
    L = np.asarray(L, dtype=np.float64)
    if L.ndim == 0:
        L = np.full(3, float(L))
    return np.ascontiguousarray(L)


def params(epsilon=1.0, sigma=1.0, mass=1.0, cutoff=2.5, skin=0.3, dt=0.005,
           rebuild_every=20, half=False, potential=0, k_spring=0.0, gamma=0.0) -> _Params:
    return _Params(epsilon, sigma, mass, cutoff, skin, dt, int(rebuild_every), int(bool(half)),
                   int(potential), 0, float(k_spring), float(gamma))


def num_threads() -> int:
    """OpenMP threads the oracle's per-atom loops use."""
    return int(_load().orc_num_threads())


def set_num_threads(k: int) -> None:
    """Threads for the oracle's later parallel loops (timing runs only)."""
    _load().orc_set_num_threads(int(k))


def cell_grid(L, r):
    """(nc[3], s[3]) with nc = floor(L / r), s = L / nc (Sec. 3.2, Fig. 1)."""
    L = _box(L)
    nc = np.zeros(3, np.int32)
    s = np.zeros(3, np.float64)
    if _load().orc_cell_grid(_dp(L), float(r), _ip(nc), _dp(s)) != 0:
        raise ValueError("box smaller than 2 (rc + skin)")
    return nc, s


def wrap(x, L):
    x = _f64(x, (-1, 3)).copy()
    _load().orc_wrap(x.shape[0], _dp(_box(L)), _dp(x))
    return x


def bin_cells(x, L, r):
    """Stable counting sort into cells.  Returns (cell_of, cell_start, cell_atoms)."""
    x = _f64(x, (-1, 3))
    nc, s = cell_grid(L, r)
    n = x.shape[0]
    ncell = int(np.prod(nc))
    cell_of = np.zeros(n, np.int32)
    start = np.zeros(ncell + 1, np.int32)
    atoms = np.zeros(n, np.int32)
    _load().orc_bin(n, _dp(x), _ip(nc), _dp(s), _ip(cell_of), _ip(start), _ip(atoms))
    return cell_of, start, atoms


def _rows(counts, lst, cap):
    return [lst[i * cap:i * cap + int(c)].copy() for i, c in enumerate(counts)]


def neighbors_brute(x, L, r, half=False, cap=256):
    """O(N^2) Verlet list: list of per-atom int32 arrays (in visit order)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    while True:
        counts = np.zeros(n, np.int32)
        lst = np.zeros(n * cap, np.int32)
        m = _load().orc_neighbors_brute(n, _dp(x), _dp(_box(L)), float(r), int(half), cap,
                                        _ip(counts), _ip(lst))
        if m <= cap:
            return _rows(counts, lst, cap)
        cap = m + 16


def neighbors_cells(x, L, r, half=False, cap=128):
    """Cell-list Verlet list of (already wrapped) positions x (Sec. 3.2, Fig. 1)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    L = _box(L)
    cell_of, start, atoms = bin_cells(x, L, r)
    nc, _ = cell_grid(L, r)
    while True:
        counts = np.zeros(n, np.int32)
        lst = np.zeros(n * cap, np.int32)
        m = _load().orc_neighbors_cells(n, _dp(x), _dp(L), _ip(nc), _ip(cell_of), _ip(start),
                                        _ip(atoms), float(r), int(half), cap, _ip(counts), _ip(lst))
        if m <= cap:
            return _rows(counts, lst, cap)
        cap = m + 16


def neighbors_cells_raw(x, L, r, half=False, cap=128):
    """Like neighbors_cells but returns (counts[n], rows[n, cap]) arrays."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    L = _box(L)
    cell_of, start, atoms = bin_cells(x, L, r)
    nc, _ = cell_grid(L, r)
    while True:
        counts = np.zeros(n, np.int32)
        lst = np.zeros(n * cap, np.int32)
        m = _load().orc_neighbors_cells(n, _dp(x), _dp(L), _ip(nc), _ip(cell_of), _ip(start),
                                        _ip(atoms), float(r), int(half), cap, _ip(counts), _ip(lst))
        if m <= cap:
            return counts, lst.reshape(n, cap)
        cap = m + 16


def neighbors_sample(x, L, r, ids, cap=256):
    """(counts[m], rows[m, cap]) of the full Verlet rows of the atoms `ids`
    (x is wrapped first), by the cell list of neighbors_cells."""
    xw = wrap(x, L)
    cell_of, start, atoms = bin_cells(xw, L, r)
    nc, _ = cell_grid(L, r)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    counts = np.zeros(ids.shape[0], np.int32)
    rows = np.zeros((ids.shape[0], cap), np.int32)
    m = _load().orc_neighbors_sample(xw.shape[0], _dp(xw), _dp(_box(L)), _ip(nc), _ip(cell_of),
                                     _ip(start), _ip(atoms), float(r), ids.shape[0],
                                     ids.ctypes.data_as(_I64), cap, _ip(counts), _ip(rows))
    if m > cap:
        raise RuntimeError(f"a row of {m} exceeds cap {cap}")
    return counts, rows


def _pack(rows):
    n = len(rows)
    cap = max(1, max((len(r) for r in rows), default=1))
    counts = np.array([len(r) for r in rows], np.int32)
    lst = np.zeros(n * cap, np.int32)
    for i, r in enumerate(rows):
        lst[i * cap:i * cap + len(r)] = r
    return cap, counts, lst


def forces_list(x, L, rows, half=False, **kw):
    """Forces over a Verlet list given as per-atom rows (Sec. 3.2 Eq. 2)."""
    x = _f64(x, (-1, 3))
    cap, counts, lst = _pack(rows)
    F = np.zeros_like(x)
    p = params(half=half, **kw)
    _load().orc_forces_list(x.shape[0], _dp(x), _dp(_box(L)), cap, _ip(counts), _ip(lst),
                            ctypes.byref(p), _dp(F))
    return F


def forces_brute(x, L, **kw):
    """The plain definition F_i = sum_{j != i, r < rc} F_LJ (minimum image)."""
    x = _f64(x, (-1, 3))
    F = np.zeros_like(x)
    p = params(**kw)
    _load().orc_forces_brute(x.shape[0], _dp(x), _dp(_box(L)), ctypes.byref(p), _dp(F))
    return F


def forces_sample(x, L, ids, **kw):
    """Plain-definition forces on the atoms `ids` only (x is wrapped first)."""
    p = params(**kw)
    xw = wrap(x, L)
    r = p.cutoff + p.skin
    cell_of, start, atoms = bin_cells(xw, L, r)
    nc, _ = cell_grid(L, r)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    F = np.zeros((ids.shape[0], 3), np.float64)
    _load().orc_forces_sample(xw.shape[0], _dp(xw), _dp(_box(L)), _ip(nc), _ip(cell_of),
                              _ip(start), _ip(atoms), ctypes.byref(p), ids.shape[0],
                              ids.ctypes.data_as(_I64), _dp(F))
    return F


def forces_sd_list(x, v, L, rows, **kw):
    """Spring-dashpot forces (Sec. 3.2 Eq. 3) over a full list; kw must give
    k_spring, gamma and sigma (the sphere diameter)."""
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    cap, counts, lst = _pack(rows)
    F = np.zeros_like(x)
    p = params(potential=1, **kw)
    _load().orc_forces_sd_list(x.shape[0], _dp(x), _dp(v), _dp(_box(L)), cap, _ip(counts),
                               _ip(lst), ctypes.byref(p), _dp(F))
    return F


def forces_sd_brute(x, v, L, **kw):
    """The plain definition of Eq. 3 over every pair (minimum image)."""
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    F = np.zeros_like(x)
    p = params(potential=1, **kw)
    _load().orc_forces_sd_brute(x.shape[0], _dp(x), _dp(v), _dp(_box(L)), ctypes.byref(p),
                                _dp(F))
    return F


def energy_sd_list(x, v, L, rows, per_atom=False, **kw):
    """(elastic PE, W) of Eq. 3 over a full list; optionally per-atom PE."""
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    cap, counts, lst = _pack(rows)
    pe = ctypes.c_double()
    w = ctypes.c_double()
    pa = np.zeros(x.shape[0], np.float64)
    p = params(potential=1, **kw)
    _load().orc_energy_sd_list(x.shape[0], _dp(x), _dp(v), _dp(_box(L)), cap, _ip(counts),
                               _ip(lst), ctypes.byref(p), ctypes.byref(pe), ctypes.byref(w),
                               _dp(pa) if per_atom else None)
    if per_atom:
        return pe.value, w.value, pa
    return pe.value, w.value


def energy_list(x, L, rows, half=False, per_atom=False, **kw):
    """(PE, W) over a list, each pair once; optionally per-atom PE."""
    x = _f64(x, (-1, 3))
    cap, counts, lst = _pack(rows)
    pe = ctypes.c_double()
    w = ctypes.c_double()
    pa = np.zeros(x.shape[0], np.float64)
    p = params(half=half, **kw)
    _load().orc_energy_list(x.shape[0], _dp(x), _dp(_box(L)), cap, _ip(counts), _ip(lst),
                            ctypes.byref(p), ctypes.byref(pe), ctypes.byref(w),
                            _dp(pa) if per_atom else None)
    if per_atom:
        return pe.value, w.value, pa
    return pe.value, w.value


def energy(x, L, **kw):
    """(PE, W) of configuration x from a fresh cell-list build."""
    p = params(**kw)
    xw = wrap(x, L)
    rows = neighbors_cells(xw, L, p.cutoff + p.skin, half=True)
    return energy_list(xw, L, rows, half=True, **kw)


def energy_atoms(x, L, rows, half=False, **kw):
    """Per-atom (PE, W) arrays over a list (each pair split half and half)."""
    x = _f64(x, (-1, 3))
    cap, counts, lst = _pack(rows)
    pe = np.zeros(x.shape[0], np.float64)
    w = np.zeros(x.shape[0], np.float64)
    p = params(half=half, **kw)
    _load().orc_energy_atoms(x.shape[0], _dp(x), _dp(_box(L)), cap, _ip(counts), _ip(lst),
                             ctypes.byref(p), _dp(pe), _dp(w))
    return pe, w


def kinetic(v, mass=1.0):
    v = _f64(v, (-1, 3))
    return float(_load().orc_kinetic(v.shape[0], _dp(v), float(mass)))


def thermo(pe, ke, w, n, L):
    """dict(pe, ke, etot, virial, temperature, pressure) of one (PE, KE, W)
    record of an n-atom box of sides L (orc_thermo)."""
    out = np.zeros(6, np.float64)
    _load().orc_thermo(float(pe), float(ke), float(w), int(n), float(np.prod(_box(L))), _dp(out))
    return dict(zip(("pe", "ke", "etot", "virial", "temperature", "pressure"), out.tolist()))


def vv_run(x, v, L, nsteps, step0=0, energies=False, **kw):
    """Velocity Verlet with the fixed rebuild schedule (Sec. 3.2 Eq. 1; Sec. 6),
    or, with rebuild_every=0, rebuilding whenever an atom has moved more than
    skin/2 since the last build.

    Returns (x, v, F[, E]) where E is (nsteps, 3) = (PE, KE, W) after each step.
    """
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    F = np.zeros_like(x)
    E = np.zeros((nsteps, 3), np.float64) if energies else None
    p = params(**kw)
    rc = _load().orc_vv_run(x.shape[0], _dp(_box(L)), ctypes.byref(p), _dp(x), _dp(v), _dp(F),
                            int(step0), int(nsteps), _dp(E) if energies else None)
    if rc != 0:
        raise RuntimeError(f"orc_vv_run failed: {rc}")
    return (x, v, F, E) if energies else (x, v, F)


def jvp(x, u, L, **kw):
    """J(x) u with J = dF/dx (the pair Hessian-vector product, sign of -H)."""
    x = _f64(x, (-1, 3))
    u = _f64(u, (-1, 3))
    out = np.zeros_like(x)
    p = params(**kw)
    rc = _load().orc_jvp(x.shape[0], _dp(_box(L)), ctypes.byref(p), _dp(x), _dp(u), _dp(out))
    if rc != 0:
        raise RuntimeError(f"orc_jvp failed: {rc}")
    return out


def traj_loss(x0, v0, L, nsteps, window, **kw):
    """Mean PE over the last `window` of `nsteps` velocity-Verlet steps."""
    x0 = _f64(x0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    out = ctypes.c_double()
    p = params(**kw)
    rc = _load().orc_traj_loss(x0.shape[0], _dp(_box(L)), ctypes.byref(p), _dp(x0), _dp(v0),
                               int(nsteps), int(window), ctypes.byref(out))
    if rc != 0:
        raise RuntimeError(f"orc_traj_loss failed: {rc}")
    return out.value


class FrozenLoss:
    """The trajectory loss with the discrete structure of a base run frozen:
    the Verlet list of each rebuild and, for each force evaluation, which
    listed pairs were inside rc.  Calling it at perturbed inputs evaluates the
    smooth branch of the loss through the base run (the unshifted cutoff makes
    the raw loss jump whenever a perturbation moves a cutoff crossing to
    another step); its finite differences are what an adjoint computes."""

    def __init__(self, x0, v0, L, nsteps, window, **kw):
        self.L, self.nsteps, self.window, self.kw = _box(L), int(nsteps), int(window), kw
        self._h = ctypes.c_void_p()
        self.base = self._run(x0, v0, 1, kw)

    def _run(self, x0, v0, mode, kw):
        x0 = _f64(x0, (-1, 3))
        v0 = _f64(v0, (-1, 3))
        out = ctypes.c_double()
        p = params(**kw)
        rc = _load().orc_traj_loss_ex(x0.shape[0], _dp(self.L), ctypes.byref(p), _dp(x0), _dp(v0),
                                      self.nsteps, self.window, ctypes.byref(out), mode,
                                      ctypes.byref(self._h))
        if rc != 0:
            raise RuntimeError(f"orc_traj_loss_ex failed: {rc}")
        return out.value

    def __call__(self, x0, v0, **overrides):
        kw = dict(self.kw)
        kw.update(overrides)
        return self._run(x0, v0, 2, kw)

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.orc_trace_free(self._h)
            self._h = ctypes.c_void_p()


def adjoint(x0, v0, L, nsteps, window, **kw):
    """(loss, dL/deps, dL/dsigma, dL/dx0, dL/dv0) by the FP64 reverse sweep."""
    x0 = _f64(x0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    loss = ctypes.c_double()
    ge = ctypes.c_double()
    gs = ctypes.c_double()
    gx = np.zeros_like(x0)
    gv = np.zeros_like(v0)
    p = params(**kw)
    rc = _load().orc_adjoint(x0.shape[0], _dp(_box(L)), ctypes.byref(p), _dp(x0), _dp(v0),
                             int(nsteps), int(window), ctypes.byref(loss), ctypes.byref(ge),
                             ctypes.byref(gs), _dp(gx), _dp(gv))
    if rc != 0:
        raise RuntimeError(f"orc_adjoint failed: {rc}")
    return loss.value, ge.value, gs.value, gx, gv
