#!/usr/bin/env python3
"""Benchmark of the LJ MD hot path: atom-timesteps/s on the 1,048,576-atom
FCC workload (64^3 unit cells, density 0.8442, T = 1.44, +-0.05 sigma jitter,
rc 2.5, skin 0.3, dt 0.005, rebuild every 20 steps).

One benchmark step = ten rebuild cycles, each binning + list build + 20
velocity-Verlet time steps (force kernel with fused integration) replayed
from one CUDA graph: 200 time steps.  value = atoms x 200 x steps / device
time of the timed region (mixed path); the FP64 path is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank advances its own copy of a single-system workload
(weak scaling, no collective on the data path); the 256-replica ensemble is
split between the ranks instead (strong scaling).  Rank 0 prints one JSON
line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2009_07400_gb300 import inputs  # noqa: E402

WORKLOAD = "fcc64_1048576"
WORKLOADS = {
    "fcc64": "fcc64_1048576",      # the benchmark configuration (default)
    "fcc128": "fcc128_8388608",    # sizing run
    "ensemble": "ensemble256",     # 256 independent replicas, one context
    "fcc80": "fcc80_2048000",      # the paper's single-GPU shape; FP64 leg: full list, 1 lane/atom
    "dem": "dem64_1048576",        # spring-dashpot contacts (Eq. 3), 1,048,576 spheres
    "adjoint": "fcc16_16384",      # differentiable rollout: 200 steps, loss window 50
    "study": "fcc64_1048576",      # design studies on the benchmark workload (run_study)
}
# the contact model's parameters for the dem workload (sigma = sphere diameter)
DEM_PARAMS = dict(sigma=1.0, cutoff=1.0, skin=0.3, dt=0.001)
DEM_K, DEM_GAMMA = 1000.0, 5.0
METRIC = "atom-timesteps/s, LJ 1M atoms, mixed-FP32 vs FP64 path at stated force error"
UNIT = "atom-timesteps/s"
STEPS_PER_CYCLE = 20                    # time steps per rebuild cycle
CYCLES_PER_STEP = 10                    # rebuild cycles per benchmark step
TIMESTEPS_PER_STEP = STEPS_PER_CYCLE * CYCLES_PER_STEP
FORCE_SRC = os.path.join(ROOT, "paper_2009_07400_gb300", "csrc", "k_force.cu")
# committed ncu summaries of the mixed force kernel on the benchmark workload,
# per list type (the kernel the autotuner picks)
PROFILE_MD = {0: os.path.join(ROOT, "profiles", "force_mixed_fcc64.md"),
              4: os.path.join(ROOT, "profiles", "force_mixed_group4_fcc64.md"),
              2: os.path.join(ROOT, "profiles", "force_mixed_group2_fcc64.md")}
LIST_NAMES = {0: "full", 1: "half", 2: "group2", 4: "group4"}


def make_workload(name, rank=0, world=1):
    """(positions, velocities, boxes, counts or None, description, seed) of a
    workload.  The ensemble is split between `world` ranks (rank's contiguous
    block of replicas, every replica generated from its own seed); the other
    workloads are one system that every rank advances on its own."""
    if name == "ensemble256":
        from paper_2009_07400_gb300 import dist as mdist
        allr = inputs.replica_ensemble(256, seed=1004)
        reps = [allr[k] for k in mdist.shard(len(allr), rank, world)]
        pos = np.concatenate([r.pos for r in reps])
        vel = np.concatenate([r.vel for r in reps])
        total = sum(r.n for r in allr)
        desc = ("256 independent periodic LJ replicas, atoms log-uniform in [500, 20000] "
                f"({total:,} in total), density U[0.70, 0.90], T U[0.8, 1.6], rc 2.5, "
                "skin 0.3, dt 0.005, rebuild every 20 steps, one context per GPU"
                + (f" (this rank: {len(reps)} replicas, {pos.shape[0]:,} atoms)" if world > 1 else ""))
        return pos, vel, [r.box for r in reps], [r.n for r in reps], desc, 1004
    s = inputs.workload(name)
    cells = {"fcc64_1048576": 64, "fcc128_8388608": 128, "fcc80_2048000": 80}[name]
    jitter = inputs.WORKLOADS[name]["jitter"]
    desc = (f"LJ 12-6 FCC {cells}^3 unit cells, {s.n:,} atoms, rho 0.8442, T 1.44, "
            f"jitter {jitter:g} sigma, rc 2.5, skin 0.3, dt 0.005, rebuild every 20 steps")
    return s.pos, s.vel, s.box, None, desc, inputs.WORKLOADS[name]["seed"]


def config_dict(n_atoms, desc, seed, timesteps_per_step=TIMESTEPS_PER_STEP):
    return {"workload": desc, "atoms": int(n_atoms), "timesteps_per_step": timesteps_per_step,
            "l2": "inputs larger than L2: the neighbour list (~0.33 GB per million atoms) "
                  "is streamed every time step; positions (16 B per atom, FP32) stay "
                  "L2-resident by design",
            "seed": seed}


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


# --------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(list_type=0):
    """DRAM bytes per launch of the mixed force kernel of `list_type` from the
    committed ncu summary, if it was taken on the current kernel source (else
    None).  Not measured in the run: ncu's counters need a profiler, and a
    number taken under one is no bench value."""
    path = PROFILE_MD.get(list_type)
    if not path or not os.path.exists(path):
        return None
    text = open(path).read()
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not h or not t:
        return None
    cur = hashlib.sha256(open(FORCE_SRC, "rb").read()).hexdigest()
    return float(t.group(1)) if h.group(1) == cur else None


def parse_tuned(text):
    """--tuned "TPA,LIST,TPA64,LIST64[,TPADW]" -> ({mixed kwargs}, {FP64
    kwargs}, {double-word kwargs or None}) or None (LIST: 0 full, 1 half, 2 / 4
    group lists; the double-word path runs full lists).  Skips the autotuner:
    under a profiler its timings include the profiler's per-launch overhead
    and it may choose another candidate than the timed run did, so profiling
    commands pin the timed run's choice."""
    if not text:
        return None
    v = [int(x) for x in text.split(",")]
    if (len(v) not in (4, 5) or v[0] not in (1, 2, 4, 8) or v[2] not in (1, 2, 4, 8)
            or v[1] not in LIST_NAMES or v[3] not in (0, 1) or (len(v) == 5 and v[4] not in (1, 2, 4, 8))):
        raise SystemExit("--tuned wants TPA,LIST,TPA64,LIST64[,TPADW] with TPA in {1,2,4,8}, "
                         "LIST in {0,1,2,4} (FP64: {0,1})")
    return (dict(threads_per_atom=v[0], list_type=v[1]),
            dict(threads_per_atom=v[2], list_type=v[3]),
            dict(threads_per_atom=v[4], list_type=0) if len(v) == 5 else None)


def algorithmic_bytes_per_atom(mean_nb, list_type, rows_per_atom=1.0):
    """DRAM bytes per atom and time step the dominant kernel must move.
    Full and group lists (force kernel with the fused velocity-Verlet
    epilogue): the 4-byte list entries (mean_nb per atom: row lengths summed
    over the rows / atoms; group lists add a byte of member bits per entry),
    4 bytes of row length per row (group rows also 4 of group table and 2 of
    member-pair mask), the FP32 position read and the next step's FP32
    position write (16 + 16), and read + write of FP64 position and velocity
    (24 B each way, 3 doubles).  Half list (force kernel alone): the list
    entries, the row length, the FP32 position read and the final force
    (16); the j-side force updates are L2 atomics.  Neighbour positions are
    gathered from L2 and are not counted."""
    if list_type == 1:
        return 4.0 * mean_nb + 4 + 16 + 16
    if list_type in (2, 4):
        return 5.0 * mean_nb + 10.0 * rows_per_atom + 16 + 16 + 2 * 24 + 2 * 24
    return 4.0 * mean_nb + 4.0 * rows_per_atom + 16 + 16 + 2 * 24 + 2 * 24


def time_cycles(ctx, steps, warmup, dist, torch, timesteps=TIMESTEPS_PER_STEP):
    """Device time of `steps` steps of `timesteps` time steps each after
    `warmup` such steps (CUDA events on the context's stream, barrier +
    synchronize on both sides)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ctx.run(timesteps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    l0 = ctx.info().kernel_launches
    start.record(stream)
    ctx.run(timesteps * steps)
    end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = start.elapsed_time(end)
    return ms, ctx.info().kernel_launches - l0


def run_gpu(args):
    import torch

    from paper_2009_07400_gb300 import build, md
    from paper_2009_07400_gb300 import dist as mdist

    rank, world, local = mdist.rank_info()
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = td
    torch.cuda.set_device(local)
    build.build()
    md.load()
    name = WORKLOADS[args.workload]
    pos, vel, box, counts, desc, seed = make_workload(name, rank, world)
    n = pos.shape[0]
    # the ensemble is split between the ranks (strong scaling); every rank
    # advances its own copy of a single-system workload (weak scaling)
    sharded = name == "ensemble256"
    # The library enqueues on the stream it is given: use one torch stream for
    # the contexts and for the CUDA events that bracket the timed region.
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream

    def make(**kw):
        return md.MDContext(pos, vel, box, counts=counts, stream=sh, **kw)

    res = {}
    pin = parse_tuned(args.tuned)
    with make(precision=md.MD_MIXED, **(pin[0] if pin else {})) as ctx:
        if pin:
            res["tuned"] = dict(pin[0], pinned=True)
        else:
            tuned = ctx.autotune(STEPS_PER_CYCLE)
            res["tuned"] = {"threads_per_atom": tuned.threads_per_atom,
                            "list_type": int(tuned.list_type)}
        res["tuned"]["cell_split"] = int(ctx.info().cell_split)
        with ClockSampler(local) as clk:
            ms, launches = time_cycles(ctx, args.steps, args.warmup, dist, torch)
        res["mixed_ms"] = ms
        res["launches"] = launches
        res["clocks"] = clk.summary()
        res["prof"] = ctx.profile(2 * STEPS_PER_CYCLE)
        res["mixed_state"] = (ctx.positions(), ctx.forces())
    # the displacement-triggered schedule (rebuild after any atom moved more
    # than skin/2) on the same workload: context for the fixed schedule
    with make(precision=md.MD_MIXED, rebuild_every=0,
              threads_per_atom=res["tuned"]["threads_per_atom"],
              list_type=res["tuned"]["list_type"]) as ctx:
        ctx.set_cell_split(res["tuned"]["cell_split"])
        disp_cycles = max(1, min(args.steps, 5))
        r0 = ctx.info().rebuilds
        ms_d, _ = time_cycles(ctx, disp_cycles, 1, dist, torch, timesteps=STEPS_PER_CYCLE)
        res["disp_ms"] = ms_d / disp_cycles
        res["disp_rebuilds"] = (ctx.info().rebuilds - r0) / ((disp_cycles + 1) * STEPS_PER_CYCLE)
    fp64_cycles = max(1, min(args.steps, 3))
    # the paper's GPU runs use full lists and one thread per atom (Sec. 6): the
    # paper-shaped workload keeps that layout for its FP64 leg
    paper_shaped = name == "fcc80_2048000"
    fp64_kw = dict(list_type=0, threads_per_atom=1) if paper_shaped else {}
    if pin and not paper_shaped:
        fp64_kw = pin[1]
    with make(precision=md.MD_FP64, **fp64_kw) as ctx:
        if paper_shaped:
            res["tuned64"] = {"threads_per_atom": 1, "list_type": 0, "paper_shaped": True}
        elif pin:
            res["tuned64"] = dict(pin[1], pinned=True)
        else:
            t64 = ctx.autotune(STEPS_PER_CYCLE)
            res["tuned64"] = {"threads_per_atom": t64.threads_per_atom,
                              "list_type": int(t64.list_type)}
        ms64, _ = time_cycles(ctx, fp64_cycles, 1, dist, torch, timesteps=STEPS_PER_CYCLE)
        res["fp64_ms"] = ms64 / fp64_cycles
        res["prof64"] = ctx.profile(STEPS_PER_CYCLE)
        res["fp64_state"] = (ctx.positions(), ctx.forces())
    # double-word pair arithmetic (MD_DW): FP64-class forces on the FP32 pipe;
    # full per-atom lists, lanes per atom from the autotuner (one lane on the
    # paper-shaped workload, as its FP64 leg)
    dw_kw = dict(threads_per_atom=1) if paper_shaped else {}
    if pin and pin[2] and not paper_shaped:
        dw_kw = pin[2]
    with make(precision=md.MD_DW, **dw_kw) as ctx:
        if paper_shaped:
            res["tuned_dw"] = {"threads_per_atom": 1, "list_type": 0, "paper_shaped": True}
        elif pin and pin[2]:
            res["tuned_dw"] = dict(pin[2], pinned=True)
        else:
            tdw = ctx.autotune(STEPS_PER_CYCLE)
            res["tuned_dw"] = {"threads_per_atom": tdw.threads_per_atom,
                               "list_type": int(tdw.list_type)}
        msdw, _ = time_cycles(ctx, fp64_cycles, 1, dist, torch, timesteps=STEPS_PER_CYCLE)
        res["dw_ms"] = msdw / fp64_cycles
        res["prof_dw"] = ctx.profile(STEPS_PER_CYCLE)
        res["dw_state"] = (ctx.positions(), ctx.forces())
    # end to end through the C ABI with host buffers, every step: the state
    # (positions and velocities) from pinned host memory -> md_set_state ->
    # one benchmark step (200 time steps) -> positions and velocities back
    # into pinned host memory.  md_set_state bins and builds for the new
    # state, so each step builds once more than the device-resident loop.
    pin_pos = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    pin_vel = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    out_pos = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    out_vel = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    pin_pos[:] = pos
    pin_vel[:] = vel
    with make(precision=md.MD_MIXED, threads_per_atom=res["tuned"]["threads_per_atom"],
              list_type=res["tuned"]["list_type"]) as ctx:
        for _ in range(2):
            ctx.set_state(pin_pos, pin_vel)
            ctx.run(TIMESTEPS_PER_STEP)
            ctx.positions(out=out_pos)
            ctx.velocities(out=out_vel)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e_steps = max(3, args.steps // 5)
        t0 = time.perf_counter()
        for _ in range(e_steps):
            ctx.set_state(pin_pos, pin_vel)
            ctx.run(TIMESTEPS_PER_STEP)
            ctx.positions(out=out_pos)
            ctx.velocities(out=out_vel)
        e2e_s = time.perf_counter() - t0
        if dist:
            dist.barrier()
    nrep = 1 if counts is None else len(counts)

    mixed_ms, fp64_ms, dw_ms, e2e_s = mdist.max_over_ranks(
        [res["mixed_ms"], res["fp64_ms"], res["dw_ms"], e2e_s], dist,
        device="cuda" if dist else None)
    n_total = n * world
    if dist and sharded:     # the ranks hold different parts of the ensemble
        t = torch.tensor([n], dtype=torch.int64, device="cuda")
        dist.all_reduce(t)
        n_total = int(t.item())
    value = n_total * TIMESTEPS_PER_STEP * args.steps / (mixed_ms / 1e3)
    fp64_value = n_total * STEPS_PER_CYCLE / (fp64_ms / 1e3)
    dw_value = n_total * STEPS_PER_CYCLE / (dw_ms / 1e3)
    e2e_value = n_total * TIMESTEPS_PER_STEP * e_steps / e2e_s
    if rank == 0:
        prof = res["prof"]
        force_ms_per_launch = prof.force_ms / max(1, prof.force_launches)
        lt = res["tuned"]["list_type"]
        bpa = algorithmic_bytes_per_atom(prof.mean_neighbors, lt, prof.rows / n)
        achieved = bpa * n / (force_ms_per_launch / 1e3) / 1e9
        peak, peak_kind = measured_peaks()
        traffic = ncu_traffic(lt) if name == WORKLOAD and lt != 1 else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": mixed_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded and world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32+f64 (mixed: FP32 pair arithmetic, Kahan sums, "
                                          "FP64 integration and reductions)",
            "data": "synthetic",
            "config": dict(config_dict(n, desc, seed), tuned=res["tuned"], replicas=nrep,
                           list=LIST_NAMES[lt]),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_source": ("dram__bytes_read.sum + dram__bytes_write.sum per "
                                            "launch from the committed ncu summary "
                                            "profiles/force_mixed_fcc64.md, taken on this "
                                            "kernel source (hash-checked); not measured in "
                                            "this run" if traffic is not None else
                                            "no ncu capture of this kernel source"),
                         "kernel": ("k_force_mixed_half" if lt == 1 else
                                    f"k_force_mixed_group<{lt}> (fused velocity-Verlet epilogue)"
                                    if lt in (2, 4) else
                                    "k_force_mixed_full (fused velocity-Verlet epilogue)"),
                         "bytes_per_atom": bpa, "list_entries_per_atom": prof.mean_neighbors,
                         "launch_ms": force_ms_per_launch, "peak_source": peak_kind},
            "phases_ms_per_timestep": {
                "force": prof.force_ms / prof.steps, "neigh": prof.neigh_ms / prof.steps,
                "other": prof.other_ms / prof.steps},
            "fp64_path": {"value": fp64_value, "ms_per_step": fp64_ms, "tuned": res["tuned64"],
                          "phases_ms_per_timestep": {
                              "force": res["prof64"].force_ms / res["prof64"].steps,
                              "neigh": res["prof64"].neigh_ms / res["prof64"].steps,
                              "other": res["prof64"].other_ms / res["prof64"].steps}},
            "dw_path": {"value": dw_value, "ms_per_step": dw_ms, "tuned": res["tuned_dw"],
                        "note": "MD_DW: pair arithmetic in double word (two FP32 numbers per "
                                "quantity) on the FP32 pipe, FP64 integration; forces within "
                                "1e-11 of the FP64 oracle (force_error.dw_max_rel)",
                        "phases_ms_per_timestep": {
                            "force": res["prof_dw"].force_ms / res["prof_dw"].steps,
                            "neigh": res["prof_dw"].neigh_ms / res["prof_dw"].steps,
                            "other": res["prof_dw"].other_ms / res["prof_dw"].steps}},
            "speedup_mixed_over_fp64": value / fp64_value,
            "speedup_dw_over_fp64": dw_value / fp64_value,
            "displacement_trigger": {
                "value": n_total * STEPS_PER_CYCLE / (res["disp_ms"] / 1e3), "unit": UNIT,
                "rebuilds_per_100_steps": 100.0 * res["disp_rebuilds"],
                "note": "mixed path, rebuild whenever an atom moved more than skin/2 since "
                        "the last binning (conditional graph node); the fixed 20-step "
                        "schedule is the headline"},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(2 * 3 * 8 * n),
                    "d2h_bytes_per_step": int(2 * 3 * 8 * n),
                    "note": "per step: positions and velocities from pinned host memory "
                            "(md_set_state, which bins and builds), 200 time steps, positions "
                            "and velocities back into pinned host memory (md_get_positions, "
                            "md_get_velocities)"},
            "gpu_launches": int(res["launches"]),
            "clocks": res["clocks"],
        }
        if not args.no_cpu_baseline:
            line.update(cpu_baseline_leg(pos, vel, box, counts, res))
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# CPU baseline leg: the FP64 oracle as it stands, on this host's cores, on a
# bounded sample of the same workload; it also states the force error of
# both GPU paths against the oracle on sampled atoms.
# --------------------------------------------------------------------------
def _systems(pos, vel, box, counts, max_atoms):
    """(pos, vel, box, offset) of the workload's systems, at most max_atoms."""
    if counts is None:
        return [(pos, vel, np.asarray(box), 0)]
    out, off, tot = [], 0, 0
    for c, b in zip(counts, box):
        if tot + c <= max_atoms or not out:
            out.append((pos[off:off + c], vel[off:off + c], np.asarray(b), off))
            tot += c
        off += c
    return out


def oracle_rate(systems, nsteps=4):
    import oracle
    oracle.build()
    atoms = t_build = t_step = 0.0
    for p, v, b, _ in systems:
        t0 = time.perf_counter()
        oracle.vv_run(p, v, b, 0)            # wrap + bin + build + one force pass
        tb = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.vv_run(p, v, b, nsteps)
        ts = (time.perf_counter() - t0 - tb) / nsteps
        t_build += max(tb - ts, 0.0)
        t_step += ts
        atoms += p.shape[0]
    rate = atoms * STEPS_PER_CYCLE / (t_build + STEPS_PER_CYCLE * t_step)
    return rate, t_step, t_build, oracle.num_threads(), int(atoms)


def cpu_baseline_leg(pos, vel, box, counts, res):
    import oracle
    systems = _systems(pos, vel, box, counts, 2_000_000 if counts is None else 60_000)
    rate, t_step, t_build, cores, atoms = oracle_rate(systems)
    what = ("the full workload" if counts is None else
            f"{len(systems)} of the replicas ({atoms:,} atoms)")
    # one core, on the paper's single-core CPU workload shape (Sec. 6: FCC
    # 32^3, 131,072 atoms), as the paper's own CPU comparison runs
    s1 = inputs.workload("fcc32_131072")
    oracle.set_num_threads(1)
    try:
        rate1, t_step1, t_build1, _, _ = oracle_rate([(s1.pos, s1.vel, s1.box, 0)])
    finally:
        oracle.set_num_threads(cores)
    out = {"cpu_baseline": {
        "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": f"FP64 C oracle (OpenMP, {cores} threads) on {what}: one list build "
                  f"({t_build:.2f} s) and 4 velocity-Verlet steps ({t_step:.3f} s each), "
                  f"rate = atoms x 20 / (build + 20 steps)",
        "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                        "sample": f"the same oracle on one thread, FCC 32^3 (131,072 atoms, the "
                                  f"paper's single-core workload): build {t_build1:.2f} s, "
                                  f"{t_step1:.3f} s per step"}}}
    rng = np.random.default_rng(0)
    errs = {}
    for key, name in (("mixed_state", "mixed_rms_rel"), ("fp64_state", "fp64_max_rel"),
                      ("dw_state", "dw_max_rel")):
        x, F = res[key]
        Fg, Fr = [], []
        per = 2048 // len(systems[:4])
        for p_r, _, b, off in systems[:4]:
            nr = p_r.shape[0]
            ids = rng.choice(nr, min(nr, per), replace=False)
            Fr.append(oracle.forces_sample(x[off:off + nr], b, ids))
            Fg.append(F[off + ids])
        Fr = np.concatenate(Fr)
        Fg = np.concatenate(Fg)
        if name == "mixed_rms_rel":
            errs[name] = float(np.sqrt(np.sum((Fg - Fr) ** 2) / np.sum(Fr ** 2)))
        else:
            frms = np.sqrt(np.mean(np.sum(Fr ** 2, axis=1)))
            sc = np.maximum(np.linalg.norm(Fr, axis=1), frms)
            errs[name] = float(np.max(np.linalg.norm(Fg - Fr, axis=1) / sc))
    errs["sample"] = "about 2048 random atoms after the timed runs, plain-definition oracle forces"
    out["force_error"] = errs
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    One step of this arm is one rebuild cycle of the workload: a call of the
    oracle's velocity-Verlet loop for 19 steps, which bins, builds the list
    and evaluates the forces once before its first step, so it holds exactly
    one list build and 20 force evaluations (the steady cycle of the 20-step
    schedule).  Steps continue from each other's final state.  The timed
    region is `steps` such calls after `warmup` untimed ones: ms_per_step x
    steps is the timed region, value = atoms x 20 x steps / its duration."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    name = WORKLOADS[args.workload]
    pos, vel, box, counts, desc, seed = make_workload(name)
    if counts is not None:     # a bounded sample of the replicas
        p, v, b, _ = _systems(pos, vel, box, counts, 60_000)[0]
    else:
        p, v, b = pos, vel, np.asarray(box)
    x, vv = p, v
    for _ in range(max(1, args.warmup)):
        x, vv, _ = oracle.vv_run(x, vv, b, STEPS_PER_CYCLE - 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x, vv, _ = oracle.vv_run(x, vv, b, STEPS_PER_CYCLE - 1)
    t_region = time.perf_counter() - t0
    value = p.shape[0] * STEPS_PER_CYCLE * args.steps / t_region
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", args.gpus)), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_region / args.steps * 1e3,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config_dict(p.shape[0], desc, seed, timesteps_per_step=STEPS_PER_CYCLE),
                           list="full", replicas=1 if counts is None else len(counts)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} rebuild cycles of "
                                       f"{'the full workload' if counts is None else 'one replica'} "
                                       f"after {max(1, args.warmup)} warm-up cycles; each cycle "
                                       "is one list build and 20 force evaluations "
                                       f"({t_region / args.steps:.2f} s per cycle)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_dem(args):
    """The contact model of Eq. 3 on a dense granular packing of 1,048,576
    spheres (mixed, double-word and FP64 paths, rebuild every 20 steps), with
    the force error of each path against the oracle on the full final state
    and the oracle's own rate on the host cores."""
    import torch

    import oracle
    from paper_2009_07400_gb300 import build, md
    torch.cuda.set_device(0)
    build.build()
    md.load()
    name = WORKLOADS["dem"]
    s = inputs.workload(name)
    n, L = s.n, s.box
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def make(prec):
        ctx = md.MDContext(s.pos, s.vel, L, stream=stream.cuda_stream, precision=prec, **DEM_PARAMS)
        ctx.set_spring_dashpot(DEM_K, DEM_GAMMA)
        return ctx

    with make(md.MD_MIXED) as ctx:
        with ClockSampler(0) as clk:
            ms, launches = time_cycles(ctx, args.steps, args.warmup, None, torch)
        prof = ctx.profile(2 * STEPS_PER_CYCLE)
    # force errors at a fixed state, the packing after one cycle of the mixed
    # path: the packing dissipates energy, and the longer it runs the closer
    # the net forces come to balance, which inflates a relative error of the
    # net forces whatever the arithmetic
    with make(md.MD_MIXED) as ctx:
        ctx.run(STEPS_PER_CYCLE)
        x, v = ctx.positions(), ctx.velocities()
        ctx.set_state(x, v)
        F_mix = ctx.forces()
    with make(md.MD_FP64) as ctx:
        c64 = max(1, min(args.steps, 3))
        ms64, _ = time_cycles(ctx, c64, 1, None, torch)
        prof64 = ctx.profile(STEPS_PER_CYCLE)
        ctx.set_state(x, v)
        F_64 = ctx.forces()
    with make(md.MD_DW) as ctx:
        cdw = max(1, min(args.steps, 3))
        msdw, _ = time_cycles(ctx, cdw, 1, None, torch)
        profdw = ctx.profile(STEPS_PER_CYCLE)
        ctx.set_state(x, v)
        F_dw = ctx.forces()
    # end to end: state from pinned host memory, one cycle, energies back
    pin_x = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    pin_v = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    pin_x[:] = s.pos
    pin_v[:] = s.vel
    with make(md.MD_MIXED) as ctx:
        ctx.set_state(pin_x, pin_v)
        ctx.run(STEPS_PER_CYCLE, energy_every=STEPS_PER_CYCLE)
        torch.cuda.synchronize()
        e_steps = max(3, args.steps // 5)
        t0 = time.perf_counter()
        for _ in range(e_steps):
            ctx.set_state(pin_x, pin_v)
            ctx.run(STEPS_PER_CYCLE, energy_every=STEPS_PER_CYCLE)
        e2e_s = time.perf_counter() - t0
    # time_cycles ran TIMESTEPS_PER_STEP time steps per benchmark step
    value = n * TIMESTEPS_PER_STEP * args.steps / (ms / 1e3)
    ok = dict(k_spring=DEM_K, gamma=DEM_GAMMA, sigma=DEM_PARAMS["sigma"])
    xw = oracle.wrap(x, L)
    rows = oracle.neighbors_cells(xw, L, DEM_PARAMS["cutoff"] + DEM_PARAMS["skin"])
    Fr = oracle.forces_sd_list(xw, v, L, rows, **ok)
    frms = np.sqrt(np.mean(np.sum(Fr ** 2, axis=1)))
    sc = np.maximum(np.linalg.norm(Fr, axis=1), frms)
    # the oracle's own rate: one build + 4 steps on the full packing
    okw = dict(potential=1, rebuild_every=STEPS_PER_CYCLE, mass=1.0, **ok,
               cutoff=DEM_PARAMS["cutoff"], skin=DEM_PARAMS["skin"], dt=DEM_PARAMS["dt"])
    t0 = time.perf_counter()
    oracle.vv_run(s.pos, s.vel, L, 0, **okw)
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.vv_run(s.pos, s.vel, L, 4, **okw)
    ts = (time.perf_counter() - t0 - tb) / 4
    cpu_rate = n * STEPS_PER_CYCLE / (max(tb - ts, 0.0) + STEPS_PER_CYCLE * ts)
    kbar = prof.mean_neighbors
    # per atom and step of the fused kernel: list entries and row length,
    # p_i and v_i (FP32 copies) read, the next p32 and v32 written, and read +
    # write of the FP64 position and velocity (24 B each way); neighbour
    # gathers come from L2
    bpa = 4.0 * kbar + 4 + 16 + 16 + 16 + 16 + 2 * 24 + 2 * 24
    launch_ms = prof.force_ms / max(1, prof.force_launches)
    peak, peak_kind = measured_peaks()
    achieved = bpa * n / (launch_ms / 1e3) / 1e9
    line = {
        "metric": "atom-timesteps/s, spring-dashpot contacts (Eq. 3), 1M spheres, mixed vs FP64 path",
        "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (mixed: FP32 pair arithmetic, FP64 integration)",
        "data": "synthetic",
        "config": {"workload": f"dense granular packing: {n:,} spheres of diameter 1, FCC with "
                               "nearest-neighbour distance 0.98 (12 contacts each), jitter 0.02, "
                               f"T 0.05, K {DEM_K:g}, gamma {DEM_GAMMA:g}, skin 0.3, dt 0.001, "
                               "rebuild every 20 steps", "atoms": n,
                   "timesteps_per_step": TIMESTEPS_PER_STEP, "seed": inputs.WORKLOADS[name]["seed"]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_force_sd_mixed (fused velocity-Verlet epilogue)",
                     "bytes_per_atom": bpa, "mean_neighbors": kbar, "launch_ms": launch_ms,
                     "peak_source": peak_kind},
        "phases_ms_per_timestep": {"force": prof.force_ms / prof.steps,
                                   "neigh": prof.neigh_ms / prof.steps,
                                   "other": prof.other_ms / prof.steps},
        "fp64_path": {"value": n * TIMESTEPS_PER_STEP * c64 / (ms64 / 1e3),
                      "phases_ms_per_timestep": {"force": prof64.force_ms / prof64.steps,
                                                 "neigh": prof64.neigh_ms / prof64.steps,
                                                 "other": prof64.other_ms / prof64.steps}},
        "dw_path": {"value": n * TIMESTEPS_PER_STEP * cdw / (msdw / 1e3),
                    "note": "double-word contact arithmetic on the FP32 pipe, FP64 integration",
                    "phases_ms_per_timestep": {"force": profdw.force_ms / profdw.steps,
                                               "neigh": profdw.neigh_ms / profdw.steps,
                                               "other": profdw.other_ms / profdw.steps}},
        "force_error": {
            "mixed_rms_rel": float(np.sqrt(np.sum((F_mix - Fr) ** 2) / np.sum(Fr ** 2))),
            "fp64_max_rel": float(np.max(np.linalg.norm(F_64 - Fr, axis=1) / sc)),
            "dw_max_rel": float(np.max(np.linalg.norm(F_dw - Fr, axis=1) / sc)),
            "sample": "every sphere, the packing after one 20-step cycle of the mixed path, "
                      "oracle list forces"},
        "e2e": {"value": n * STEPS_PER_CYCLE * e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(2 * 3 * 8 * n), "d2h_bytes_per_step": 24},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"FP64 C oracle (OpenMP, {oracle.num_threads()} threads) on the "
                                   f"full packing: one list build ({max(tb - ts, 0.0):.2f} s) and 4 "
                                   f"steps ({ts:.3f} s each), rate = atoms x 20 / (build + 20 steps)"},
    }
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """The differentiable rollout (16,384 atoms, 200 velocity-Verlet steps,
    loss = mean PE over the last 50, checkpoints every 10): md_adjoint's
    forward + reverse sweep timed for both paths against the forward run
    alone, with the gradients compared to the oracle's FP64 reverse sweep,
    whose time on the host cores is the CPU baseline."""
    import torch

    import oracle
    from paper_2009_07400_gb300 import build, md
    torch.cuda.set_device(0)
    build.build()
    md.load()
    name = WORKLOADS["adjoint"]
    s = inputs.workload(name)
    n = s.n
    nsteps, window, ckpt = 200, 50, 10
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    res = {}
    for label, prec in (("mixed", md.MD_MIXED), ("fp64", md.MD_FP64), ("dw", md.MD_DW)):
        with md.MDContext(s.pos, s.vel, s.box, stream=stream.cuda_stream, precision=prec) as ctx:
            # lanes per atom of the force kernels tuned as in the main bench
            # (md_adjoint walks full per-atom lists: another choice falls back)
            tuned = ctx.autotune(20)
            tune = dict(threads_per_atom=tuned.threads_per_atom, list_type=int(tuned.list_type))
            for _ in range(max(1, args.warmup)):
                out = ctx.adjoint(nsteps, window, ckpt)
            torch.cuda.synchronize()
            reps = max(1, min(args.steps, 5))
            t0 = time.perf_counter()
            for _ in range(reps):
                out = ctx.adjoint(nsteps, window, ckpt)
            t_adj = (time.perf_counter() - t0) / reps
            x0, v0 = ctx.positions(), ctx.velocities()
        with md.MDContext(s.pos, s.vel, s.box, stream=stream.cuda_stream, precision=prec,
                          **tune) as ctx:
            ctx.run(nsteps)
            ctx.set_state(s.pos, s.vel)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.run(nsteps)
            torch.cuda.synchronize()
            t_fwd = time.perf_counter() - t0
        res[label] = (out, t_adj, t_fwd, tune)
    t0 = time.perf_counter()
    ref = oracle.adjoint(s.pos, s.vel, s.box, nsteps, window)
    t_orc = time.perf_counter() - t0

    def errs(out):
        loss, ge, gs, gx, gv = out
        return {"loss_rel": abs(loss - ref[0]) / abs(ref[0]),
                "d_eps_rel": abs(ge - ref[1]) / abs(ref[1]),
                "d_sigma_rel": abs(gs - ref[2]) / abs(ref[2]),
                "d_x0_rel_norm": float(np.linalg.norm(gx - ref[3]) / np.linalg.norm(ref[3])),
                "d_v0_rel_norm": float(np.linalg.norm(gv - ref[4]) / np.linalg.norm(ref[4]))}

    out_m, t_m, f_m, tune_m = res["mixed"]
    out_d, t_d, f_d, tune_d = res["fp64"]
    out_w, t_w, f_w, tune_w = res["dw"]
    rate = lambda t: n * nsteps / t                          # noqa: E731
    line = {
        "metric": "atom-timesteps/s of the differentiated LJ rollout (forward + reverse sweep)",
        "value": rate(t_m), "unit": UNIT, "n_gpus": 1, "steps": max(1, min(args.steps, 5)),
        "warmup": args.warmup, "ms_per_step": t_m * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed forward, FP64 adjoint accumulation)", "data": "synthetic",
        "config": {"workload": f"LJ FCC 16^3, {n:,} atoms, rho 0.8442, T 1.44, {nsteps} steps, "
                               f"loss = mean PE over the last {window}, checkpoints every {ckpt}, "
                               "gradients w.r.t. epsilon, sigma, x0, v0", "atoms": n,
                   "timesteps_per_step": nsteps, "seed": inputs.WORKLOADS[name]["seed"],
                   "tuned": {"mixed": tune_m, "fp64": tune_d, "dw": tune_w}},
        "adjoint_over_forward": {"mixed": t_m / f_m, "fp64": t_d / f_d, "dw": t_w / f_w},
        "fp64_path": {"value": rate(t_d), "ms_per_step": t_d * 1e3},
        "dw_path": {"value": rate(t_w), "ms_per_step": t_w * 1e3,
                    "note": "double-word forward, recompute and reverse pair terms"},
        "gradient_error_vs_oracle": {"mixed": errs(out_m), "fp64": errs(out_d), "dw": errs(out_w)},
        "cpu_baseline": {"value": rate(t_orc), "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"the oracle's FP64 reverse sweep of the same rollout "
                                   f"({t_orc:.2f} s, OpenMP {oracle.num_threads()} threads)"},
        "timing": "host wall clock around md_adjoint (it synchronises: loss and gradients "
                  "are returned in host memory)",
    }
    print(json.dumps(line), flush=True)


def _study_context(md, s, stream, **kw):
    ctx = md.MDContext(s.pos, s.vel, s.box, stream=stream, precision=md.MD_MIXED, **kw)
    ctx.run(STEPS_PER_CYCLE)              # a rebuild cycle: the steady state
    return ctx


def run_cellorder_child(tile):
    """One cell order (cells numbered in tiles of `tile` cells per edge; the
    library uses 2): build that library, time the 1M-atom mixed step (per
    phase with md_profile, and a graph-replayed 200-step run with CUDA
    events) and print one JSON object."""
    import torch

    from paper_2009_07400_gb300 import build, md
    torch.cuda.set_device(0)
    md.load(build.build(cell_tile=tile))
    s = inputs.workload(WORKLOAD)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"cell_tile": tile}
    with _study_context(md, s, stream.cuda_stream, list_type=0, threads_per_atom=1) as ctx:
        ctx.run(2 * STEPS_PER_CYCLE)
        p = ctx.profile(4 * STEPS_PER_CYCLE)
        out["force_us"] = 1e3 * p.force_ms / p.steps
        out["neigh_us_per_step"] = 1e3 * p.neigh_ms / p.steps
        ms, _ = time_cycles(ctx, 3, 1, None, torch)
        out["step_us"] = 1e3 * ms / (3 * TIMESTEPS_PER_STEP)
        ids = np.random.default_rng(0).choice(s.n, 512, replace=False)
        out["force_sample"] = ctx.forces()[ids].tolist()
    print(json.dumps(out), flush=True)


def run_study(args):
    """Design studies behind the library's choices, on the 1,048,576-atom
    benchmark workload (mixed path), each against the library's own choice on
    the same state:
      * force-kernel variants (md_study_force_variant, full per-atom list,
        one lane per atom, forces only): gathered-position layouts (AoS, the
        library's; SoA; AoSoA), the tile neighbourhood staged in shared
        memory, and gathers through the texture path;
      * list types: the per-atom full list against lists shared by groups of
        2 and 4 atoms (md_profile per phase);
      * cell orders: libraries built with cell tiles of 1 (z fastest), 2 (the
        library's) and 4 cells per edge, each timed in its own process;
      * cell size of the list build: whole cells (the library's default)
        against cells split into octants (md_set_cell_split), on this
        workload and on the 256-replica ensemble (small boxes, cells up to
        ~1.3 rc + skin).
    Prints one JSON line."""
    import torch

    from paper_2009_07400_gb300 import build, md
    torch.cuda.set_device(0)
    build.build()
    md.load()
    s = inputs.workload(WORKLOAD)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    reps = max(5, args.steps)
    names = {0: "AoS float4 (library)", 1: "SoA", 2: "AoSoA (blocks of 4)",
             3: "2x2x2-cell tiles, 4x4x4-cell neighbourhood in shared memory",
             4: "the same staged by TMA bulk copies (one per cell)",
             5: "AoS float4 gathers through the texture path",
             6: "half of the gathers through the texture path"}
    variants = {}
    with _study_context(md, s, stream.cuda_stream, list_type=0, threads_per_atom=1) as ctx:
        F = {}
        for v in (0, 1, 2, 3, 4, 5, 6):
            times = [ctx.study_force_variant(v, reps)[0] for _ in range(3)]
            F[v] = ctx.study_force_variant(v, 1, forces=True)[1]
            variants[names[v]] = {"us_per_launch": min(times), "runs": times}
        for v in (1, 2, 3, 4, 5, 6):
            d = F[v] - F[0]
            variants[names[v]]["max_abs_force_diff_vs_library"] = float(np.abs(d).max())
            variants[names[v]]["rms_rel_vs_library"] = float(np.sqrt(np.sum(d ** 2) / np.sum(F[0] ** 2)))
    lists = {}
    for lt, nm in ((0, "per-atom full"), (2, "groups of 2"), (4, "groups of 4")):
        with _study_context(md, s, stream.cuda_stream, list_type=lt, threads_per_atom=1) as ctx:
            ctx.run(2 * STEPS_PER_CYCLE)
            p = ctx.profile(4 * STEPS_PER_CYCLE)
            ms, _ = time_cycles(ctx, 2, 1, None, torch)
            lists[nm] = {"force_us": 1e3 * p.force_ms / p.steps,
                         "neigh_us_per_step": 1e3 * p.neigh_ms / p.steps,
                         "list_entries_per_atom": p.mean_neighbors,
                         "step_us": 1e3 * ms / (2 * TIMESTEPS_PER_STEP)}
    splits = {}
    ens = inputs.replica_ensemble(256, seed=1004)
    systems = {WORKLOAD: (s.pos, s.vel, s.box, None),
               "ensemble256": (np.concatenate([r.pos for r in ens]), np.concatenate([r.vel for r in ens]),
                               [r.box for r in ens], [r.n for r in ens])}
    for wname, (pos, vel, box, counts) in systems.items():
        splits[wname] = {}
        with md.MDContext(pos, vel, box, counts=counts, stream=stream.cuda_stream,
                          precision=md.MD_MIXED, list_type=0, threads_per_atom=1) as ctx:
            for split in (0, 1):
                ctx.set_cell_split(split)
                ctx.run(2 * STEPS_PER_CYCLE)
                p = ctx.profile(4 * STEPS_PER_CYCLE)
                ms, _ = time_cycles(ctx, 2, 1, None, torch)
                splits[wname]["octants" if split else "whole cells (library)"] = {
                    "neigh_us_per_step": 1e3 * p.neigh_ms / p.steps,
                    "force_us": 1e3 * p.force_ms / p.steps,
                    "step_us": 1e3 * ms / (2 * TIMESTEPS_PER_STEP)}
    orders = {}
    for tile in (1, 2, 4):
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cellorder-child", str(tile)],
                           capture_output=True, text=True, timeout=1800)
        if r.returncode != 0:
            raise SystemExit(f"cell-order child {tile} failed:\n{r.stderr[-3000:]}")
        orders[tile] = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    ref = np.array(orders[2].pop("force_sample"))
    for tile in (1, 4):
        f = np.array(orders[tile].pop("force_sample"))
        orders[tile]["rms_rel_force_vs_tile2"] = float(np.sqrt(np.sum((f - ref) ** 2) / np.sum(ref ** 2)))
    line = {"study": "design choices of the mixed force path, 1,048,576-atom FCC liquid "
                     "(rho 0.8442, T 1.44, jitter 0.05), full lists unless stated",
            "force_kernel_variants": variants, "list_types": lists,
            "cell_orders": {f"tiles of {t} cells per edge" + (" (library)" if t == 2 else ""): o
                            for t, o in orders.items()},
            "cell_split": splits,
            "timing": "CUDA events on the context's stream; variants: best of 3 runs of "
                      f"{reps} launches each"}
    print(json.dumps(line), flush=True)


def run_ncu_case(which, pin=None):
    """Create the workload's context and run 2 cycles: 1 first drift, then
    per cycle 19 fused steps, a rebuild (binning kernels + build) and the
    20th fused step.  `dem`: the contact model on the 1M-sphere packing
    (mixed path, force and integration kernels per step).  pin: the --tuned
    lanes per atom and list type of the mixed (or FP64) context."""
    import torch

    from paper_2009_07400_gb300 import build, md
    torch.cuda.set_device(0)
    build.build()
    if which in ("dem", "dem_dw"):
        s = inputs.workload(WORKLOADS["dem"])
        prec = md.MD_MIXED if which == "dem" else md.MD_DW
        with md.MDContext(s.pos, s.vel, s.box, precision=prec, **DEM_PARAMS) as ctx:
            ctx.set_spring_dashpot(DEM_K, DEM_GAMMA)
            ctx.run(2 * STEPS_PER_CYCLE)
        torch.cuda.synchronize()
        return
    s = inputs.workload(WORKLOAD)
    prec = {"mixed": md.MD_MIXED, "fp64": md.MD_FP64, "dw": md.MD_DW}[which]
    kw = ((pin[0] if which == "mixed" else pin[1]) if pin and which != "dw" else {})
    with md.MDContext(s.pos, s.vel, s.box, precision=prec, **kw) as ctx:
        ctx.run(2 * STEPS_PER_CYCLE)
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="fcc64", choices=sorted(WORKLOADS),
                    help="fcc64: the 1,048,576-atom benchmark (default); fcc128: the "
                         "8,388,608-atom sizing run; ensemble: 256 replicas; fcc80: the "
                         "paper's 2,048,000-atom GPU shape; dem: 1,048,576 spheres with "
                         "the contact model of Eq. 3")
    ap.add_argument("--tuned", metavar="TPA,LIST,TPA64,LIST64[,TPADW]",
                    help="skip the autotuner and use these lanes per atom and list "
                         "types for the mixed and FP64 legs (for profiling commands)")
    ap.add_argument("--cellorder-child", type=int, choices=[1, 2, 4], help=argparse.SUPPRESS)
    ap.add_argument("--ncu-case", choices=["mixed", "fp64", "dw", "dem", "dem_dw"],
                    help="only build the workload and run 2 rebuild cycles (a short, "
                         "fixed launch sequence for an ncu capture); prints nothing")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.cellorder_child:
        run_cellorder_child(args.cellorder_child)
    elif args.ncu_case:
        run_ncu_case(args.ncu_case, parse_tuned(args.tuned))
    elif args.workload == "study":
        if args.impl == "native":
            run_study(args)
        else:
            print(json.dumps({"impl": "reference", "unavailable": "the design studies compare "
                              "GPU kernels with each other; the oracle arm covers the "
                              "forward workloads"}), flush=True)
    elif args.workload == "adjoint":
        if args.impl == "native":
            run_adjoint(args)
        else:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the "
                              "forward workloads; the adjoint line carries its own "
                              "cpu_baseline"}), flush=True)
    elif args.workload == "dem":
        if args.impl == "native":
            run_dem(args)
        else:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the "
                              "Lennard-Jones workloads; the dem line carries its own "
                              "cpu_baseline"}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
