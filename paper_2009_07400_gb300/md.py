"""Thin ctypes binding of the C ABI in ``include/md.h`` (same names).

Argument marshalling only: every step of the MD path runs in the CUDA
library ``libmdgb300.so``.  There is no fallback; if the library is missing
or cannot be loaded the import of a context raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmdgb300.so")

MD_OK = 0
ERRORS = {
    -1: "MD_ERR_INVAL", -2: "MD_ERR_BOX_TOO_SMALL", -3: "MD_ERR_NOMEM", -4: "MD_ERR_CUDA",
    -5: "MD_ERR_NL_OVERFLOW", -6: "MD_ERR_TIMEOUT", -7: "MD_ERR_NONFINITE",
    -8: "MD_ERR_BADPOS", -9: "MD_ERR_STATE",
}
MD_FP64, MD_MIXED, MD_DW = 0, 1, 2
MD_LIST_FULL, MD_LIST_HALF, MD_LIST_GROUP2, MD_LIST_GROUP4 = 0, 1, 2, 4
(MD_ERR_INVAL, MD_ERR_BOX_TOO_SMALL, MD_ERR_NOMEM, MD_ERR_CUDA, MD_ERR_NL_OVERFLOW,
 MD_ERR_TIMEOUT, MD_ERR_NONFINITE, MD_ERR_BADPOS, MD_ERR_STATE) = range(-1, -10, -1)

# Every exported entry point of the ABI (checked by the load test).
ABI_SYMBOLS = [
    "md_create", "md_create_batch", "md_destroy", "md_last_error", "md_set_state",
    "md_bin_cells", "md_build_neighbors", "md_compute_forces", "md_integrate", "md_energy",
    "md_run", "md_get_positions", "md_get_velocities", "md_get_forces", "md_get_cells",
    "md_get_neighbors", "md_get_info", "md_autotune", "md_set_capacity", "md_profile",
    "md_set_lj", "md_adjoint", "md_energy_sums_static", "md_create_device",
    "md_set_state_device", "md_get_positions_device", "md_get_velocities_device",
    "md_get_forces_device", "md_set_spring_dashpot", "md_set_step",
    "md_set_adjoint_precision", "md_thermo", "md_adjoint_device", "md_study_force_variant",
    "md_set_cell_split",
]


class MDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class md_box(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class md_params(ctypes.Structure):
    _fields_ = [("epsilon", ctypes.c_double), ("sigma", ctypes.c_double),
                ("mass", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("skin", ctypes.c_double), ("dt", ctypes.c_double),
                ("rebuild_every", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("list_type", ctypes.c_int32), ("threads_per_atom", ctypes.c_int32)]


class md_phase_times(ctypes.Structure):
    _fields_ = [("force_ms", ctypes.c_double), ("neigh_ms", ctypes.c_double),
                ("other_ms", ctypes.c_double), ("force_launches", ctypes.c_int64),
                ("neigh_launches", ctypes.c_int64), ("other_launches", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("mean_neighbors", ctypes.c_double),
                ("rows", ctypes.c_int64)]


class md_thermo_rec(ctypes.Structure):
    _fields_ = [("pe", ctypes.c_double), ("ke", ctypes.c_double), ("etot", ctypes.c_double),
                ("virial", ctypes.c_double), ("temperature", ctypes.c_double),
                ("pressure", ctypes.c_double)]


class md_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nrep", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("list_type", ctypes.c_int32),
                ("threads_per_atom", ctypes.c_int32), ("list_capacity", ctypes.c_int32),
                ("max_neighbors", ctypes.c_int32), ("ncells", ctypes.c_int64),
                ("step", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("rebuilds", ctypes.c_int64), ("cell_split", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)


def load(path: str | None = None):
    """Loads libmdgb300.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library {p} is missing; run paper_2009_07400_gb300.build")
            lib = ctypes.CDLL(p)
            ctx = ctypes.c_void_p
            sig = {
                "md_create": [ctypes.POINTER(md_box), ctypes.POINTER(md_params), ctypes.c_int64,
                              _D, _D, _P, ctypes.POINTER(ctx)],
                "md_create_batch": [ctypes.c_int32, ctypes.POINTER(md_box),
                                    ctypes.POINTER(md_params), _I64, _D, _D, _P,
                                    ctypes.POINTER(ctx)],
                "md_destroy": [ctx],
                "md_last_error": [ctx],
                "md_set_state": [ctx, _D, _D],
                "md_bin_cells": [ctx],
                "md_build_neighbors": [ctx],
                "md_compute_forces": [ctx],
                "md_integrate": [ctx, ctypes.c_int32],
                "md_energy": [ctx, _D, _D, _D],
                "md_run": [ctx, ctypes.c_int64, ctypes.c_int32, _D],
                "md_get_positions": [ctx, _D],
                "md_get_velocities": [ctx, _D],
                "md_get_forces": [ctx, _D],
                "md_get_cells": [ctx, _I32, _I32],
                "md_get_neighbors": [ctx, _I32, _I32, ctypes.c_int32],
                "md_get_info": [ctx, ctypes.POINTER(md_info)],
                "md_autotune": [ctx, ctypes.c_int32, ctypes.POINTER(md_params)],
                "md_set_capacity": [ctx, ctypes.c_int32],
                "md_profile": [ctx, ctypes.c_int64, ctypes.POINTER(md_phase_times)],
                "md_set_lj": [ctx, ctypes.c_double, ctypes.c_double],
                "md_adjoint": [ctx, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _D, _D, _D,
                               _D, _D],
                "md_energy_sums_static": [ctypes.c_int64, _P, _P, _P, ctypes.c_double, _P, _P],
                "md_create_device": [ctypes.POINTER(md_box), ctypes.POINTER(md_params),
                                     ctypes.c_int64, _P, _P, _P, ctypes.POINTER(ctx)],
                "md_set_state_device": [ctx, _P, _P],
                "md_get_positions_device": [ctx, _P],
                "md_get_velocities_device": [ctx, _P],
                "md_get_forces_device": [ctx, _P],
                "md_set_spring_dashpot": [ctx, ctypes.c_double, ctypes.c_double],
                "md_set_step": [ctx, ctypes.c_int64],
                "md_set_adjoint_precision": [ctx, ctypes.c_int32],
                "md_thermo": [ctx, _D, ctypes.c_int64, ctypes.POINTER(md_thermo_rec)],
                "md_adjoint_device": [ctx, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _D,
                                      _D, _D, _P, _P],
                "md_study_force_variant": [ctx, ctypes.c_int32, ctypes.c_int32, _D, _D],
                "md_set_cell_split": [ctx, ctypes.c_int32],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.md_destroy.restype = None
            lib.md_last_error.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def energy_sums_static(n, pe_atom_ptr, w_atom_ptr, vel_ptr, mass, out3_ptr, stream=None):
    """md_energy_sums_static on device pointers (ints); raises MDError."""
    lib = load()
    rc = lib.md_energy_sums_static(int(n), ctypes.c_void_p(pe_atom_ptr), ctypes.c_void_p(w_atom_ptr),
                                   ctypes.c_void_p(vel_ptr), float(mass),
                                   ctypes.c_void_p(out3_ptr),
                                   ctypes.c_void_p(int(stream)) if stream else None)
    if rc != MD_OK:
        raise MDError(rc, lib.md_last_error(None).decode())


def _dev3(a):
    """A contiguous CUDA float64 (n, 3) tensor, or TypeError."""
    import torch
    if not isinstance(a, torch.Tensor) or not a.is_cuda or a.dtype != torch.float64:
        raise TypeError("expected a CUDA float64 tensor")
    if a.dim() != 2 or a.shape[1] != 3 or not a.is_contiguous():
        raise TypeError("expected a contiguous n x 3 tensor")
    return a


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(n, 3)
    return a


def make_params(epsilon=1.0, sigma=1.0, mass=1.0, cutoff=2.5, skin=0.3, dt=0.005,
                rebuild_every=20, precision=MD_FP64, half_list=False, threads_per_atom=0,
                list_type=None):
    """md_params; list_type (MD_LIST_*) wins over the older half_list flag.
    precision: MD_FP64, MD_MIXED (FP32 pairs) or MD_DW (pairs in double word,
    full lists only)."""
    lt = int(list_type) if list_type is not None else (MD_LIST_HALF if half_list else MD_LIST_FULL)
    return md_params(epsilon, sigma, mass, cutoff, skin, dt, int(rebuild_every), int(precision),
                     lt, int(threads_per_atom))


class MDContext:
    """One md_ctx: a periodic system (or a batch of replicas) on the GPU."""

    def __init__(self, pos, vel, box, stream=None, counts=None, **params):
        lib = load()
        self._lib = lib
        self.params = make_params(**params)
        if counts is None:
            pos = np.asarray(pos, np.float64).reshape(-1, 3)
            boxes = [np.broadcast_to(np.asarray(box, np.float64), (3,))]
            counts = [pos.shape[0]]
        else:
            boxes = [np.broadcast_to(np.asarray(b, np.float64), (3,)) for b in box]
        self.counts = np.ascontiguousarray(counts, dtype=np.int64)
        self.n = int(self.counts.sum())
        self.nrep = len(self.counts)
        pos = _f64(pos, self.n)
        vel = _f64(vel, self.n)
        self._boxes = [np.array(b, np.float64) for b in boxes]
        barr = (md_box * self.nrep)(*[md_box(*map(float, b)) for b in boxes])
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(int(stream)) if stream else None
        rc = lib.md_create_batch(self.nrep, barr, ctypes.byref(self.params),
                                 self.counts.ctypes.data_as(_I64), pos.ctypes.data_as(_D),
                                 vel.ctypes.data_as(_D), st, ctypes.byref(h))
        if rc != MD_OK:
            raise MDError(rc, lib.md_last_error(None).decode())
        self._h = h

    @classmethod
    def from_device(cls, pos, vel, box, stream=None, **params):
        """A single-system context from CUDA float64 tensors (n x 3) without a
        host copy (md_create_device).  The context runs on `stream` (a
        torch.cuda.Stream; a new one if None), which first waits for the
        current stream, where pos and vel were produced."""
        import torch
        pos, vel = _dev3(pos), _dev3(vel)
        if pos.shape != vel.shape:
            raise ValueError("pos and vel differ in shape")
        self = cls.__new__(cls)
        self._lib = load()
        self.params = make_params(**params)
        self.counts = np.array([pos.shape[0]], np.int64)
        self.n = int(pos.shape[0])
        self.nrep = 1
        self._tstream = stream if stream is not None else torch.cuda.Stream(device=pos.device)
        self._tstream.wait_stream(torch.cuda.current_stream(pos.device))
        bx = np.array(np.broadcast_to(np.asarray(box, np.float64), (3,)))
        self._boxes = [bx]
        b = md_box(*map(float, bx))
        h = ctypes.c_void_p()
        rc = self._lib.md_create_device(ctypes.byref(b), ctypes.byref(self.params), self.n,
                                        ctypes.c_void_p(pos.data_ptr()),
                                        ctypes.c_void_p(vel.data_ptr()),
                                        ctypes.c_void_p(self._tstream.cuda_stream), ctypes.byref(h))
        if rc != MD_OK:
            raise MDError(rc, self._lib.md_last_error(None).decode())
        self._h = h
        return self

    # -- helpers --------------------------------------------------------------
    def _check(self, rc):
        if rc != MD_OK:
            raise MDError(rc, self._lib.md_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.md_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the ABI --------------------------------------------------------------
    def set_state(self, pos, vel):
        pos = _f64(pos, self.n)
        vel = _f64(vel, self.n)
        self._check(self._lib.md_set_state(self._h, pos.ctypes.data_as(_D), vel.ctypes.data_as(_D)))

    def set_state_device(self, pos, vel):
        """md_set_state_device from CUDA float64 tensors (n x 3)."""
        import torch
        pos, vel = _dev3(pos), _dev3(vel)
        if tuple(pos.shape) != (self.n, 3) or tuple(vel.shape) != (self.n, 3):
            raise ValueError("expected n x 3 tensors")
        self._before_device_call(torch)
        self._check(self._lib.md_set_state_device(self._h, ctypes.c_void_p(pos.data_ptr()),
                                                  ctypes.c_void_p(vel.data_ptr())))

    def _before_device_call(self, torch):
        ts = getattr(self, "_tstream", None)
        if ts is not None:
            ts.wait_stream(torch.cuda.current_stream(ts.device))
        else:
            torch.cuda.current_stream().synchronize()

    def _get3_device(self, fn, out):
        import torch
        if out is None:
            out = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        out = _dev3(out)
        if tuple(out.shape) != (self.n, 3):
            raise ValueError("expected an n x 3 tensor")
        self._before_device_call(torch)
        self._check(fn(self._h, ctypes.c_void_p(out.data_ptr())))
        ts = getattr(self, "_tstream", None)
        if ts is not None:
            torch.cuda.current_stream(ts.device).wait_stream(ts)
        else:
            torch.cuda.synchronize()
        return out

    def positions_device(self, out=None):
        """Positions into a CUDA float64 tensor (n x 3), caller order."""
        return self._get3_device(self._lib.md_get_positions_device, out)

    def velocities_device(self, out=None):
        return self._get3_device(self._lib.md_get_velocities_device, out)

    def forces_device(self, out=None):
        return self._get3_device(self._lib.md_get_forces_device, out)

    def bin_cells(self):
        self._check(self._lib.md_bin_cells(self._h))

    def build_neighbors(self):
        self._check(self._lib.md_build_neighbors(self._h))

    def compute_forces(self):
        self._check(self._lib.md_compute_forces(self._h))

    def integrate(self, phase):
        self._check(self._lib.md_integrate(self._h, int(phase)))

    def energy(self):
        """(PE, KE, W) arrays of length nrep (FP64)."""
        pe = np.zeros(self.nrep)
        ke = np.zeros(self.nrep)
        w = np.zeros(self.nrep)
        self._check(self._lib.md_energy(self._h, pe.ctypes.data_as(_D), ke.ctypes.data_as(_D),
                                        w.ctypes.data_as(_D)))
        return pe, ke, w

    def run(self, nsteps, energy_every=0):
        """Advance nsteps; with energy_every > 0 returns (nsteps//every, nrep, 3)."""
        if energy_every > 0:
            out = np.zeros((nsteps // energy_every, self.nrep, 3))
            self._check(self._lib.md_run(self._h, int(nsteps), int(energy_every),
                                         out.ctypes.data_as(_D)))
            return out
        self._check(self._lib.md_run(self._h, int(nsteps), 0, None))
        return None

    def _get3(self, fn, out=None):
        """n x 3 doubles from fn into `out` (a C-contiguous float64 array, e.g.
        one in pinned host memory) or a new array."""
        if out is None:
            out = np.zeros((self.n, 3))
        elif (out.dtype != np.float64 or out.shape != (self.n, 3)
              or not out.flags["C_CONTIGUOUS"]):
            raise ValueError("out must be a C-contiguous float64 n x 3 array")
        self._check(fn(self._h, out.ctypes.data_as(_D)))
        return out

    def positions(self, out=None):
        return self._get3(self._lib.md_get_positions, out)

    def velocities(self, out=None):
        return self._get3(self._lib.md_get_velocities, out)

    def forces(self, out=None):
        return self._get3(self._lib.md_get_forces, out)

    def cells(self):
        """(cell_start per replica incl. end, cell_atoms replica-local ids)."""
        info = self.info()
        start = np.zeros(info.ncells + self.nrep, np.int32)
        atoms = np.zeros(self.n, np.int32)
        self._check(self._lib.md_get_cells(self._h, start.ctypes.data_as(_I32),
                                           atoms.ctypes.data_as(_I32)))
        return start, atoms

    def _row_cap(self):
        """A row capacity that holds every exact row of the current list (a
        member of a group list can have up to its group row plus the other
        members)."""
        inf = self.info()
        return max(4, inf.list_capacity, inf.max_neighbors) + 8

    def neighbors(self):
        """Per-atom rows (caller order, replica-local ids) of the current list."""
        cap = self._row_cap()
        counts = np.zeros(self.n, np.int32)
        rows = np.zeros(self.n * cap, np.int32)
        self._check(self._lib.md_get_neighbors(self._h, counts.ctypes.data_as(_I32),
                                               rows.ctypes.data_as(_I32), cap))
        return [rows[i * cap:i * cap + counts[i]].copy() for i in range(self.n)]

    def neighbors_raw(self, cap=None):
        """(counts[n], rows[n, cap]) of the current list, caller order; cap
        defaults to one that holds every row (MD_ERR_INVAL if a row exceeds a
        given cap)."""
        cap = cap or self._row_cap()
        counts = np.zeros(self.n, np.int32)
        rows = np.zeros((self.n, cap), np.int32)
        self._check(self._lib.md_get_neighbors(self._h, counts.ctypes.data_as(_I32),
                                               rows.ctypes.data_as(_I32), cap))
        return counts, rows

    def profile(self, nsteps) -> md_phase_times:
        out = md_phase_times()
        self._check(self._lib.md_profile(self._h, int(nsteps), ctypes.byref(out)))
        return out

    def set_lj(self, epsilon, sigma):
        self._check(self._lib.md_set_lj(self._h, float(epsilon), float(sigma)))

    def set_spring_dashpot(self, k_spring, gamma):
        """Contact model of Eq. 3 (spheres of diameter params.sigma)."""
        self._check(self._lib.md_set_spring_dashpot(self._h, float(k_spring), float(gamma)))

    def adjoint(self, nsteps, window, ckpt_every=10):
        """(loss, dL/deps, dL/dsigma, dL/dx0 (n x 3), dL/dv0 (n x 3))."""
        loss = ctypes.c_double()
        ge = ctypes.c_double()
        gs = ctypes.c_double()
        gx = np.zeros((self.n, 3))
        gv = np.zeros((self.n, 3))
        self._check(self._lib.md_adjoint(self._h, int(nsteps), int(window), int(ckpt_every),
                                         ctypes.byref(loss), ctypes.byref(ge), ctypes.byref(gs),
                                         gx.ctypes.data_as(_D), gv.ctypes.data_as(_D)))
        return loss.value, ge.value, gs.value, gx, gv

    def adjoint_device(self, nsteps, window, ckpt_every=10, g_x0=None, g_v0=None):
        """md_adjoint_device: (loss, dL/deps, dL/dsigma, dL/dx0, dL/dv0) with the
        two n x 3 gradients in CUDA float64 tensors (new ones if None)."""
        import torch
        if g_x0 is None:
            g_x0 = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        if g_v0 is None:
            g_v0 = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        g_x0, g_v0 = _dev3(g_x0), _dev3(g_v0)
        if tuple(g_x0.shape) != (self.n, 3) or tuple(g_v0.shape) != (self.n, 3):
            raise ValueError("expected n x 3 tensors")
        loss = ctypes.c_double()
        ge = ctypes.c_double()
        gs = ctypes.c_double()
        self._before_device_call(torch)
        self._check(self._lib.md_adjoint_device(self._h, int(nsteps), int(window), int(ckpt_every),
                                                ctypes.byref(loss), ctypes.byref(ge),
                                                ctypes.byref(gs), ctypes.c_void_p(g_x0.data_ptr()),
                                                ctypes.c_void_p(g_v0.data_ptr())))
        return loss.value, ge.value, gs.value, g_x0, g_v0

    def study_force_variant(self, variant, reps=10, forces=False):
        """md_study_force_variant: (microseconds per launch, forces or None)."""
        us = ctypes.c_double()
        F = np.zeros((self.n, 3)) if forces else None
        self._check(self._lib.md_study_force_variant(self._h, int(variant), int(reps), ctypes.byref(us),
                                                     F.ctypes.data_as(_D) if forces else None))
        return us.value, F

    def set_adjoint_precision(self, precision):
        """Precision of the reverse sweep's pair terms (MD_FP64, MD_MIXED, or
        MD_DW on a double-word context)."""
        self._check(self._lib.md_set_adjoint_precision(self._h, int(precision)))

    def set_cell_split(self, split):
        """1: the list build scans half-size cells (each cell's atoms ordered
        by octant); 0: whole cells.  Rebins and rebuilds."""
        self._check(self._lib.md_set_cell_split(self._h, int(split)))

    def set_capacity(self, cap):
        self._check(self._lib.md_set_capacity(self._h, int(cap)))

    def set_step(self, step):
        """Step counter of the rebuild schedule (for resuming a saved run)."""
        self._check(self._lib.md_set_step(self._h, int(step)))

    def thermo(self, energies=None):
        """md_thermo: per-replica pe, ke, etot, virial, temperature and
        pressure from (PE, KE, W) triples (md_run's energy log, any leading
        shape) or, with None, from the current state.  Arrays of shape
        energies.shape[:-1] (or (nrep,))."""
        if energies is None:
            shape, arg, nrec = (self.nrep,), None, 1
        else:
            e = np.ascontiguousarray(energies, np.float64)
            if e.shape[-1] != 3 or e.size % (3 * self.nrep) != 0:
                raise ValueError("expected (..., nrep, 3) energy records")
            shape, nrec = e.shape[:-1], e.size // (3 * self.nrep)
            arg = e.ctypes.data_as(_D)
        out = (md_thermo_rec * (nrec * self.nrep))()
        self._check(self._lib.md_thermo(self._h, arg, nrec, out))
        raw = np.ctypeslib.as_array(ctypes.cast(out, ctypes.POINTER(ctypes.c_double)),
                                    shape=(nrec * self.nrep * 6,)).reshape(shape + (6,)).copy()
        names = ("pe", "ke", "etot", "virial", "temperature", "pressure")
        return {k: raw[..., q] for q, k in enumerate(names)}

    def info(self) -> md_info:
        inf = md_info()
        self._check(self._lib.md_get_info(self._h, ctypes.byref(inf)))
        return inf

    def autotune(self, steps=20) -> md_params:
        out = md_params()
        self._check(self._lib.md_autotune(self._h, int(steps), ctypes.byref(out)))
        return out
