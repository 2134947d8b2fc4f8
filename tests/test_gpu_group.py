"""Lists shared by groups of 2 or 4 atoms of a cell (MD_LIST_GROUP2/4, mixed
path) against the FP64 oracle, through the C ABI.

A group's row is the union of its members' rows (built with an FP32 test
whose margin covers the FP64 criterion), so the parity object stays the
per-atom row: md_get_neighbors filters each member's candidates (the group
row plus the other members) with the exact FP64 criterion on the device, and
the result must equal the oracle's cell-list rows as sorted sets, bit for
bit.  Forces and energies carry the mixed path's tolerances (RMS relative
force error <= 1e-5).
"""
import numpy as np
import pytest

from paper_2009_07400_gb300 import inputs

pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3
GROUPS = [2, 4]


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


def sorted_rows(counts, rows):
    big = np.iinfo(np.int32).max
    width = max(1, int(counts.max()))
    out = np.full((counts.shape[0], width), big, np.int64)
    mask = np.arange(width)[None, :] < counts[:, None]
    out[mask] = rows[:, :width][mask]
    out.sort(axis=1)
    return out


def assert_rows_exact(orc, ctx, x, L, o=0, n=None):
    c_g, r_g = ctx.neighbors_raw()
    n = c_g.shape[0] if n is None else n
    c_g, r_g = c_g[o:o + n], r_g[o:o + n]
    c_o, r_o = orc.neighbors_cells_raw(orc.wrap(x, L), L, RC + SKIN, cap=1024)
    assert np.array_equal(c_g, c_o)
    assert np.array_equal(sorted_rows(c_g, r_g), sorted_rows(c_o, r_o))


def liquid(orc, n_cells=7, steps=60, seed=3):
    s = inputs.fcc_system(n_cells, jitter=0.05, seed=seed)
    x, v, _ = orc.vv_run(s.pos, s.vel, s.box, steps)
    return inputs.System(x, v, s.box, seed)


def band_system(seed=5, L=(30.0, 31.0, 29.0)):
    """Pairs within 1e-15 .. 1e-5 of the list radius (and exactly on it): the
    FP32 union test must keep them for the FP64 filter to decide."""
    rng = np.random.default_rng(seed)
    L = np.array(L)
    rs = RC + SKIN
    a = rng.uniform(0, 1, size=(120, 3)) * L
    u = rng.normal(size=(120, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    delta = rng.choice([-1, 1], 120) * 10.0 ** rng.uniform(-15, -5, 120)
    b = a + rs * (1 + delta)[:, None] * u
    ax = np.array([[3.0, 4.0, 5.0], [3.0 + rs, 4.0, 5.0]])
    pos = np.concatenate([a, b, ax]) % L
    return inputs.System(pos, np.zeros_like(pos), L, seed)


def system_of(orc, case):
    if case == "fcc8":
        return inputs.fcc_system(8, seed=1001)
    if case == "jitter7":
        return inputs.fcc_system(7, jitter=0.1, seed=8)
    if case == "nc2":
        return inputs.uniform_box(400, (5.7, 5.7, 5.7), seed=9)
    if case == "aniso":
        return inputs.uniform_box(900, (5.7, 9.0, 12.3), seed=10)
    if case == "band":
        return band_system()
    if case == "band_wide":
        return band_system(seed=6, L=(8.39, 5.75, 30.0))
    if case == "ragged":
        return inputs.replica_system(2999, 0.82, 1.3, seed=12)
    return liquid(orc)


@pytest.mark.parametrize("g", GROUPS)
@pytest.mark.parametrize("case", ["fcc8", "jitter7", "nc2", "aniso", "band", "band_wide",
                                  "liquid", "ragged"])
def test_group_rows_exact(md, orc, case, g):
    """Exact per-atom rows from a group list: cells with 1..G members in their
    last group, boxes with 2 cells per edge (each periodic image visited
    once), pairs on the edge of the list radius; with whole and split cells."""
    s = system_of(orc, case)
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, list_type=g) as ctx:
        assert ctx.info().list_type == g
        assert_rows_exact(orc, ctx, s.pos, s.box)
        ctx.set_cell_split(1)          # groups then follow the octant order of a cell
        assert_rows_exact(orc, ctx, s.pos, s.box)


@pytest.mark.parametrize("g", GROUPS)
@pytest.mark.parametrize("case", ["jitter7", "liquid", "ragged", "aniso"])
def test_group_forces_and_energies(md, orc, case, g):
    s = system_of(orc, case)
    if case == "aniso":                          # uniform points overlap: a soft liquid instead
        s = inputs.replica_system(1500, 0.75, 1.0, seed=31)
    xw = orc.wrap(s.pos, s.box)
    rows = orc.neighbors_cells(xw, s.box, RC + SKIN)
    Fr = orc.forces_list(xw, s.box, rows)
    pe, w = orc.energy_list(xw, s.box, orc.neighbors_cells(xw, s.box, RC + SKIN, half=True),
                            half=True)
    ke = orc.kinetic(s.vel)
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, list_type=g) as ctx:
        assert rms_rel(ctx.forces(), Fr) <= 1e-5
        gpe, gke, gw = ctx.energy()
        assert gpe[0] == pytest.approx(pe, rel=1e-6)
        assert gke[0] == pytest.approx(ke, rel=1e-13)
        assert abs(gw[0] - w) <= 1e-5 * abs(2 * ke + w)


@pytest.mark.parametrize("g", GROUPS)
def test_group_run_vs_oracle_and_full_list(md, orc, g):
    """100 steps of the 131,072-atom workload: total energy against the
    oracle (mixed tolerance, 1e-5 per atom before decorrelation) and against
    the per-atom full list of the same path."""
    s = inputs.workload("fcc32_131072")
    x_ref, v_ref, _, E_ref = orc.vv_run(s.pos, s.vel, s.box, 100, energies=True)
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, list_type=g) as ctx:
        E = ctx.run(100, energy_every=20)
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED) as ctx:
        Ef = ctx.run(100, energy_every=20)
    for k in range(5):
        e_ref = E_ref[20 * k + 19, 0] + E_ref[20 * k + 19, 1]
        assert abs(E[k, 0, 0] + E[k, 0, 1] - e_ref) / s.n <= 1e-5
        assert abs(E[k, 0, 0] + E[k, 0, 1] - Ef[k, 0, 0] - Ef[k, 0, 1]) / s.n <= 1e-5


@pytest.mark.parametrize("g", GROUPS)
def test_group_split_runs_and_overflow(md, orc, g):
    """Splitting a run changes no bit (fixed summation order: each lane's
    Kahan sums, then a fixed butterfly); a group row that overflows at an
    in-run rebuild is grown and the run resumes there with the same result.
    The capacity is set to the largest group row of the initial lattice
    (rounded up to 16), which the melting lattice outgrows."""
    kw = dict(precision=md.MD_MIXED, list_type=g)
    s = liquid(orc, n_cells=6)
    with md.MDContext(s.pos, s.vel, s.box, **kw) as a, \
            md.MDContext(s.pos, s.vel, s.box, **kw) as b:
        a.run(57)
        b.run(13)
        b.run(20)
        b.run(24)
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.velocities(), b.velocities())
    s = inputs.workload("fcc8_2048")
    with md.MDContext(s.pos, s.vel, s.box, **kw) as a, \
            md.MDContext(s.pos, s.vel, s.box, **kw) as c:
        c.set_capacity(c.info().max_neighbors)
        cap0 = c.info().list_capacity
        assert cap0 % 16 == 0 and cap0 >= c.info().max_neighbors
        a.run(100)
        c.run(100)
        assert c.info().list_capacity > cap0
        assert np.array_equal(a.positions(), c.positions())
        assert np.array_equal(a.velocities(), c.velocities())


@pytest.mark.parametrize("g", GROUPS)
def test_group_batched_replicas(md, orc, g):
    """Replicas of uneven sizes in one context: groups never straddle cells
    or replicas; per replica, exact rows and forces against the oracle."""
    reps = inputs.replica_ensemble(6, seed=77, n_min=500, n_max=3000)
    pos = np.concatenate([r.pos for r in reps])
    vel = np.concatenate([r.vel for r in reps])
    counts = [r.n for r in reps]
    with md.MDContext(pos, vel, [r.box for r in reps], counts=counts, precision=md.MD_MIXED,
                      list_type=g) as ctx:
        ctx.run(20)
        X, F = ctx.positions(), ctx.forces()
        o = 0
        for r in reps:
            x = X[o:o + r.n]
            assert_rows_exact(orc, ctx, x, r.box, o, r.n)
            xw = orc.wrap(x, r.box)
            Fr = orc.forces_list(xw, r.box, orc.neighbors_cells(xw, r.box, RC + SKIN))
            assert rms_rel(F[o:o + r.n], Fr) <= 1e-5
            o += r.n


@pytest.mark.parametrize("g", GROUPS)
def test_group_displacement_trigger(md, orc, g):
    """rebuild_every = 0 with a group list: the run follows the oracle's
    fresh-list run to the mixed path's accuracy."""
    s = liquid(orc, n_cells=7)
    x_ref, _, _, E_ref = orc.vv_run(s.pos, s.vel, s.box, 120, rebuild_every=1, energies=True)
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, rebuild_every=0,
                      list_type=g) as ctx:
        E = ctx.run(120, energy_every=40)
        x = ctx.positions()
    d = x - x_ref
    d -= s.box * np.round(d / s.box)
    assert np.abs(d).max() < 1e-5
    for k in range(3):
        e_ref = E_ref[40 * k + 39, 0] + E_ref[40 * k + 39, 1]
        assert abs(E[k, 0, 0] + E[k, 0, 1] - e_ref) / s.n < 1e-5


@pytest.mark.parametrize("g", GROUPS)
def test_group_full_size(md, orc, g):
    """The 1,048,576-atom benchmark workload after one graph-replayed rebuild
    cycle, in the launch shape the bench times: every row exact, forces on
    sampled atoms."""
    s = inputs.workload("fcc64_1048576")
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, list_type=g) as ctx:
        ctx.run(20)
        x = ctx.positions()
        assert_rows_exact(orc, ctx, x, s.box)
        ids = np.random.default_rng(0).choice(s.n, 4096, replace=False)
        Fr = orc.forces_sample(x, s.box, ids)
        assert rms_rel(ctx.forces()[ids], Fr) <= 1e-5


def test_group_list_rules(md, orc):
    """Group lists need the mixed path; the adjoint and the contact model
    switch to per-atom full lists (the adjoint switches back and gives the
    full list's bits), and the tuner may choose a group list."""
    s = liquid(orc, n_cells=5)
    with pytest.raises(md.MDError) as e:
        md.MDContext(s.pos, s.vel, s.box, precision=md.MD_FP64, list_type=4)
    assert e.value.code == md.MD_ERR_INVAL
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED, list_type=4) as a, \
            md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED) as b:
        ga = a.adjoint(20, 10, 10)
        gb = b.adjoint(20, 10, 10)
        assert a.info().list_type == 4
        assert ga[0] == gb[0] and np.array_equal(ga[3], gb[3])
        a.set_spring_dashpot(0.0, 0.0)
        assert a.info().list_type == 0
    with md.MDContext(s.pos, s.vel, s.box, precision=md.MD_MIXED) as ctx:
        chosen = ctx.autotune(steps=20)
        assert chosen.list_type in (0, 1, 2, 4)
