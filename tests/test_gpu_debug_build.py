"""The bounds-checked build (MD_DEBUG_CHECKS=1) stands in for a memory
checker: every gathered or stored index of the kernels is checked on the
device, and a bad one raises an error flag (MD_ERR_STATE) instead of
touching memory.  Here it runs the main paths (per-atom and group lists,
replicas, the contact model, the adjoint, the force-kernel studies, the
split-cell build, the double-word path with its contact model and adjoint) with no check firing and must agree bit for bit with the
normal build on every deterministic path (the half-list paths add forces
with atomics, so only their completion counts)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, sys
import numpy as np
sys.path.insert(0, %(root)r)
from paper_2009_07400_gb300 import inputs, md
md.load(sys.argv[1])

def h(*arrays):
    m = hashlib.sha256()
    for a in arrays:
        m.update(np.ascontiguousarray(a).tobytes())
    return m.hexdigest()[:16]

out = []
s = inputs.workload("fcc8_2048")
for prec in (md.MD_FP64, md.MD_MIXED):
    for half in (False, True):
        with md.MDContext(s.pos, s.vel, s.box, precision=prec, half_list=half) as c:
            E = c.run(60, energy_every=20)
            cnt, rows = c.neighbors_raw()
            # half lists add the j-side forces with atomics, whose order (and
            # so the last bits) varies from run to run: only the run counts
            out.append("half-ok" if half else h(c.positions(), c.velocities(), c.forces(), E, cnt))
    with md.MDContext(s.pos, s.vel, s.box, precision=prec, rebuild_every=0) as c:
        c.run(60)
        out.append(h(c.positions(), c.velocities()))
reps = inputs.replica_ensemble(3, seed=5, n_min=500, n_max=2000)
pos = np.concatenate([r.pos for r in reps]); vel = np.concatenate([r.vel for r in reps])
with md.MDContext(pos, vel, [r.box for r in reps], counts=[r.n for r in reps],
                  precision=md.MD_MIXED) as c:
    c.run(40)
    out.append(h(c.positions()))
rng = np.random.default_rng(3)
L = np.array([8.0, 8.5, 9.0])
x = rng.uniform(0, 1, (600, 3)) * L
v = rng.normal(size=(600, 3))
for prec in (md.MD_FP64, md.MD_MIXED, md.MD_DW):
    with md.MDContext(x, v, L, sigma=1.0, cutoff=1.0, skin=0.3, dt=0.001, precision=prec) as c:
        c.set_spring_dashpot(200.0, 2.0)
        c.run(60)
        out.append(h(c.positions(), c.velocities()))
# lists shared by groups of atoms (their own build, force kernel and row
# decode), a batch of replicas with them, and the force-kernel studies
for g in (2, 4):
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, list_type=g) as c:
        E = c.run(60, energy_every=20)
        cnt, rows = c.neighbors_raw()
        out.append(h(c.positions(), c.velocities(), c.forces(), E, cnt))
with md.MDContext(pos, vel, [r.box for r in reps], counts=[r.n for r in reps],
                  precision=md.MD_MIXED, list_type=4) as c:
    c.run(40)
    out.append(h(c.positions()))
with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED) as c:
    c.set_cell_split(1)          # binning keys per octant, the split build
    E = c.run(60, energy_every=20)
    cnt, rows = c.neighbors_raw()
    out.append(h(c.positions(), c.velocities(), c.forces(), E, cnt))
with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_DW) as c:   # double-word pairs
    E = c.run(60, energy_every=20)
    out.append(h(c.positions(), c.velocities(), c.forces(), E))
with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, threads_per_atom=1) as c:
    c.run(20)
    out.append(h(*[c.study_force_variant(v, 1, forces=True)[1] for v in range(7)]))
s4 = inputs.fcc_system(4, jitter=0.05, seed=2)
for prec in (md.MD_FP64, md.MD_DW):
    with md.MDContext(s4.pos, s4.vel, s4.box, precision=prec) as c:
        loss, ge, gs, gx, gv = c.adjoint(20, 10, 10)
        out.append(h(np.array([loss, ge, gs]), gx, gv))
print(" ".join(out))
"""


def test_debug_build_agrees_and_stays_silent():
    from paper_2009_07400_gb300 import build
    release = build.build()
    debug = build.build(debug=True)
    script = SCRIPT % {"root": ROOT}
    res = {}
    for name, lib in (("release", release), ("debug", debug)):
        r = subprocess.run([sys.executable, "-c", script, lib], capture_output=True, text=True,
                           timeout=900)
        assert r.returncode == 0, f"{name}: {r.stderr[-3000:]}"
        res[name] = r.stdout.split()
    assert len(res["release"]) == 18
    assert res["debug"] == res["release"]
