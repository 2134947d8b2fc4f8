"""Spring-dashpot contact model (Sec. 3.2, Eq. 3) on the GPU against the
oracle: forces and energies on the same state, trajectories, and the
closed-form restitution of a two-sphere collision."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIG, SKIN = 1.0, 0.3


@pytest.fixture(scope="module")
def md():
    from paper_2009_07400_gb300 import build
    build.build()
    from paper_2009_07400_gb300 import md as m
    m.load()
    return m


def dense(seed=3, n=600, L=(8.0, 8.5, 9.0)):
    """Overlapping spheres (packing fraction ~0.75) with random velocities."""
    rng = np.random.default_rng(seed)
    L = np.array(L)
    return rng.uniform(0, 1, (n, 3)) * L, rng.normal(size=(n, 3)), L


def sd_ctx(md, x, v, L, k, g, **kw):
    ctx = md.MDContext(x, v, L, sigma=SIG, cutoff=SIG, skin=SKIN, **kw)
    ctx.set_spring_dashpot(k, g)
    return ctx


def rel_rms(F, Fr):
    return np.sqrt(np.sum((F - Fr) ** 2) / np.sum(Fr ** 2))


@pytest.mark.parametrize("half", [False, True])
def test_forces_and_energy(md, orc, half):
    x, v, L = dense()
    xw = orc.wrap(x, L)
    rows = orc.neighbors_cells(xw, L, SIG + SKIN)
    ok = dict(k_spring=500.0, gamma=3.0, sigma=SIG)
    Fr = orc.forces_sd_list(xw, v, L, rows, **ok)
    pe_r, w_r = orc.energy_sd_list(xw, v, L, rows, **ok)
    for precision, tol in ((md.MD_FP64, 1e-12), (md.MD_MIXED, 1e-5)):
        with sd_ctx(md, x, v, L, 500.0, 3.0, precision=precision, half_list=half) as ctx:
            assert ctx.info().list_type == 0        # contacts use full lists
            F = ctx.forces()
            assert rel_rms(F, Fr) < tol
            pe, ke, w = (q[0] for q in ctx.energy())
            assert pe == pytest.approx(pe_r, rel=max(tol, 1e-12))
            assert w == pytest.approx(w_r, rel=max(10 * tol, 1e-11))
            assert ke == pytest.approx(0.5 * np.sum(v ** 2), rel=1e-13)
    # K = gamma = 0: no force at all (the paper's static setting)
    with sd_ctx(md, x, v, L, 0.0, 0.0, precision=md.MD_FP64) as ctx:
        assert np.all(ctx.forces() == 0.0)


@pytest.mark.parametrize("every", [20, 0])
def test_trajectory_fp64(md, orc, every):
    """300 steps of a dissipative dense gas: FP64 path against the oracle's
    velocity Verlet (dashpot on the half-step velocities)."""
    x, v, L = dense(seed=9, n=400)
    kw = dict(k_spring=200.0, gamma=2.0, sigma=SIG, cutoff=SIG, skin=SKIN, dt=0.001)
    xr, vr, Fr, Er = orc.vv_run(x, v, L, 300, energies=True, potential=1,
                                rebuild_every=every if every else 0, **kw)
    with sd_ctx(md, x, v, L, 200.0, 2.0, precision=md.MD_FP64, dt=0.001, rebuild_every=every) as ctx:
        E = ctx.run(300, energy_every=100)
        d = np.mod(ctx.positions() - xr + L / 2, L) - L / 2
        assert np.abs(d).max() < 1e-9
        assert np.abs(ctx.velocities() - vr).max() < 1e-8
    for k in range(3):
        et = E[k, 0, 0] + E[k, 0, 1]
        er = Er[100 * k + 99, 0] + Er[100 * k + 99, 1]
        assert et == pytest.approx(er, rel=1e-10)
    assert E[2, 0, 0] + E[2, 0, 1] < 0.8 * (E[0, 0, 0] + E[0, 0, 1])   # the gas cools


@pytest.mark.parametrize("split", [0, 1])
def test_trajectory_mixed(md, orc, split):
    """Mixed path against the oracle's run; also with split cells (the
    binning then orders each cell's spheres by octant and reorders the FP32
    velocity copies with them)."""
    x, v, L = dense(seed=9, n=400)
    kw = dict(k_spring=200.0, gamma=2.0, sigma=SIG, cutoff=SIG, skin=SKIN, dt=0.001)
    xr, vr, _, Er = orc.vv_run(x, v, L, 200, energies=True, potential=1, **kw)
    with sd_ctx(md, x, v, L, 200.0, 2.0, precision=md.MD_MIXED, dt=0.001) as ctx:
        ctx.set_cell_split(split)
        E = ctx.run(200, energy_every=200)
        d = np.mod(ctx.positions() - xr + L / 2, L) - L / 2
        assert np.abs(d).max() < 1e-4
    et = E[0, 0, 0] + E[0, 0, 1]
    er = Er[199, 0] + Er[199, 1]
    assert abs(et - er) / abs(er) < 1e-4


def test_restitution_on_gpu(md):
    """Two spheres meeting head-on leave with e = exp(-zeta pi/sqrt(1-zeta^2))
    times the approach speed (damped oscillator of the overlap, mu = m/2)."""
    k, g, u, dt = 1000.0, 5.0, 1.0, 1e-5
    mu = 0.5
    zeta = g / (2.0 * math.sqrt(mu * k))
    e = math.exp(-zeta * math.pi / math.sqrt(1.0 - zeta ** 2))
    wd = math.sqrt(k / mu) * math.sqrt(1.0 - zeta ** 2)
    L = np.array([20.0, 20.0, 20.0])
    x = np.array([[10.0, 10.0, 10.0], [10.0 + SIG + 0.25 * u * dt, 10.0, 10.0]])
    v = np.array([[0.5 * u, 0.0, 0.0], [-0.5 * u, 0.0, 0.0]])
    steps = int(1.5 * math.pi / wd / dt)
    with sd_ctx(md, x, v, L, k, g, precision=md.MD_FP64, dt=dt) as ctx:
        ctx.run(steps)
        vn = ctx.velocities()
    assert abs((vn[1, 0] - vn[0, 0]) / u - e) < 1e-4
    assert abs(vn[:, 0].sum()) < 1e-12


def test_contact_model_argument_checks(md):
    x, v, L = dense(n=50)
    with md.MDContext(x, v, L, sigma=SIG, cutoff=0.9, skin=SKIN) as ctx:
        with pytest.raises(md.MDError) as e:
            ctx.set_spring_dashpot(10.0, 1.0)                 # cutoff < sigma
        assert e.value.code == md.MD_ERR_INVAL
    with sd_ctx(md, x, v, L, 10.0, 1.0) as ctx:
        with pytest.raises(md.MDError):
            ctx.set_spring_dashpot(-1.0, 0.0)
        with pytest.raises(md.MDError) as e:
            ctx.adjoint(20, 10, 10)
        assert e.value.code == md.MD_ERR_INVAL
        ctx.set_lj(1.0, 1.0)                                  # back to Lennard-Jones
        ctx.forces()


def test_batched_packings_with_displacement_trigger(md, orc):
    """Three independent packings of different sizes in one context, the
    displacement-triggered schedule, FP64: each replica follows its own
    oracle run (dashpot on the half-step velocities)."""
    systems = [dense(seed=s, n=n, L=L) for s, n, L in
               ((11, 300, (7.0, 7.0, 7.5)), (12, 450, (8.0, 8.0, 8.0)), (13, 200, (6.0, 6.5, 7.0)))]
    pos = np.concatenate([x for x, _, _ in systems])
    vel = np.concatenate([v for _, v, _ in systems])
    kw = dict(sigma=SIG, cutoff=SIG, skin=SKIN, dt=0.001)
    with md.MDContext(pos, vel, [L for _, _, L in systems], counts=[x.shape[0] for x, _, _ in systems],
                      precision=md.MD_FP64, rebuild_every=0, **kw) as ctx:
        ctx.set_spring_dashpot(300.0, 1.5)
        ctx.run(150)
        xg = ctx.positions()
        assert ctx.info().rebuilds > 1
    o = 0
    for x, v, L in systems:
        xr, _, _ = orc.vv_run(x, v, L, 150, potential=1, k_spring=300.0, gamma=1.5,
                              rebuild_every=0, **kw)
        d = np.mod(xg[o:o + x.shape[0]] - xr + L / 2, L) - L / 2
        assert np.abs(d).max() < 1e-9
        o += x.shape[0]


@pytest.mark.parametrize("every", [20, 0])
def test_mixed_fused_step_split_runs_are_bitwise_equal(md, every):
    """The mixed contact step is one fused kernel that also writes the next
    FP32 velocity copies; copies are regenerated only where something else
    changed v (the first drift of a run, a final lone kick).  A run split
    into pieces, with energies logged and an eager profiled stretch, must
    give the same bits as one run, on both rebuild schedules."""
    x, v, L = dense(seed=21, n=500)
    kw = dict(precision=md.MD_MIXED, dt=0.001, rebuild_every=every)
    with sd_ctx(md, x, v, L, 300.0, 2.5, **kw) as ctx:
        ctx.run(75)
        ref = (ctx.positions(), ctx.velocities(), ctx.forces())
    with sd_ctx(md, x, v, L, 300.0, 2.5, **kw) as ctx:
        ctx.run(7, energy_every=3)
        ctx.run(20)
        ctx.profile(21)
        ctx.run(27, energy_every=27)
        got = (ctx.positions(), ctx.velocities(), ctx.forces())
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_mixed_batched_packings_with_displacement_trigger(md, orc):
    """Three packings in one context on the mixed fused step with the
    displacement-triggered schedule, against the oracle."""
    systems = [dense(seed=s, n=n, L=L) for s, n, L in
               ((31, 300, (7.0, 7.0, 7.5)), (32, 450, (8.0, 8.0, 8.0)), (33, 200, (6.0, 6.5, 7.0)))]
    pos = np.concatenate([x for x, _, _ in systems])
    vel = np.concatenate([v for _, v, _ in systems])
    kw = dict(sigma=SIG, cutoff=SIG, skin=SKIN, dt=0.001)
    with md.MDContext(pos, vel, [L for _, _, L in systems], counts=[x.shape[0] for x, _, _ in systems],
                      precision=md.MD_MIXED, rebuild_every=0, **kw) as ctx:
        ctx.set_spring_dashpot(300.0, 1.5)
        ctx.run(150)
        xg = ctx.positions()
        assert ctx.info().rebuilds > 1
    o = 0
    for x, v, L in systems:
        xr, _, _ = orc.vv_run(x, v, L, 150, potential=1, k_spring=300.0, gamma=1.5,
                              rebuild_every=0, **kw)
        d = np.mod(xg[o:o + x.shape[0]] - xr + L / 2, L) - L / 2
        assert np.abs(d).max() < 1e-4
        o += x.shape[0]


def test_mixed_state_changes_refresh_velocity_copies(md, orc):
    """New velocities from set_state, a direct half kick (md_integrate) and a
    switch of the contact constants must reach the dashpot term: each case
    against the oracle's forces on the same state."""
    x, v, L = dense(seed=41, n=400)
    ok = dict(k_spring=250.0, gamma=4.0, sigma=SIG)
    with sd_ctx(md, x, v, L, 250.0, 4.0, precision=md.MD_MIXED, dt=0.001) as ctx:
        ctx.run(30)
        v2 = -ctx.velocities()                   # reverse every velocity
        x2 = ctx.positions()
        ctx.set_state(x2, v2)
        xw = orc.wrap(x2, L)
        rows = orc.neighbors_cells(xw, L, SIG + SKIN)
        assert rel_rms(ctx.forces(), orc.forces_sd_list(xw, v2, L, rows, **ok)) < 1e-5
        ctx.run(10)
        ctx.integrate(1)                         # half kick + drift outside a run
        xi, vi = ctx.positions(), ctx.velocities()
        xw = orc.wrap(xi, L)
        rows = orc.neighbors_cells(xw, L, SIG + SKIN)
        assert rel_rms(ctx.forces(), orc.forces_sd_list(xw, vi, L, rows, **ok)) < 1e-5
        ctx.set_spring_dashpot(250.0, 8.0)
        ok8 = dict(ok, gamma=8.0)
        assert rel_rms(ctx.forces(), orc.forces_sd_list(xw, vi, L, rows, **ok8)) < 1e-5


def test_dw_forces_and_energy(md, orc):
    """Double-word contact forces and energies on the same state as the FP64
    path: within 1e-11 (the FP64 path: 1e-12; the mixed path: 1e-5)."""
    x, v, L = dense()
    xw = orc.wrap(x, L)
    rows = orc.neighbors_cells(xw, L, SIG + SKIN)
    ok = dict(k_spring=500.0, gamma=3.0, sigma=SIG)
    Fr = orc.forces_sd_list(xw, v, L, rows, **ok)
    pe_r, w_r = orc.energy_sd_list(xw, v, L, rows, **ok)
    for lanes in (1, 4):
        with sd_ctx(md, x, v, L, 500.0, 3.0, precision=md.MD_DW, threads_per_atom=lanes) as ctx:
            F = ctx.forces()
            err = rel_rms(F, Fr)
            print("double-word contact forces, RMS relative error:", err)
            assert err < 1e-11
            pe, ke, w = (q[0] for q in ctx.energy())
            assert pe == pytest.approx(pe_r, rel=1e-11)
            assert w == pytest.approx(w_r, rel=1e-10)
            assert ke == pytest.approx(0.5 * np.sum(v ** 2), rel=1e-13)


@pytest.mark.parametrize("every", [20, 0])
def test_trajectory_dw(md, orc, every):
    """300 steps of the dissipative dense gas on the double-word fused step
    (velocity copies split into high and low parts): the FP64 path's bar."""
    x, v, L = dense(seed=9, n=400)
    kw = dict(k_spring=200.0, gamma=2.0, sigma=SIG, cutoff=SIG, skin=SKIN, dt=0.001)
    xr, vr, Fr, Er = orc.vv_run(x, v, L, 300, energies=True, potential=1,
                                rebuild_every=every if every else 0, **kw)
    with sd_ctx(md, x, v, L, 200.0, 2.0, precision=md.MD_DW, dt=0.001, rebuild_every=every) as ctx:
        E = ctx.run(300, energy_every=100)
        d = np.mod(ctx.positions() - xr + L / 2, L) - L / 2
        assert np.abs(d).max() < 1e-9
        assert np.abs(ctx.velocities() - vr).max() < 1e-8
    for k in range(3):
        et = E[k, 0, 0] + E[k, 0, 1]
        er = Er[100 * k + 99, 0] + Er[100 * k + 99, 1]
        assert et == pytest.approx(er, rel=1e-10)


def test_dw_fused_step_split_runs_are_bitwise_equal(md):
    """The double-word contact step writes the next velocity copies (both
    parts); a run split into pieces with energies and a profiled stretch
    gives the same bits as one run."""
    x, v, L = dense(seed=21, n=500)
    kw = dict(precision=md.MD_DW, dt=0.001)
    with sd_ctx(md, x, v, L, 300.0, 2.5, **kw) as ctx:
        ctx.run(75)
        ref = (ctx.positions(), ctx.velocities(), ctx.forces())
    with sd_ctx(md, x, v, L, 300.0, 2.5, **kw) as ctx:
        ctx.run(7, energy_every=3)
        ctx.run(20)
        ctx.profile(21)
        ctx.run(27, energy_every=27)
        got = (ctx.positions(), ctx.velocities(), ctx.forces())
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_dw_batched_packings_and_restitution(md, orc):
    """Three packings in one double-word context with the displacement
    trigger against the oracle, and the two-sphere restitution."""
    systems = [dense(seed=s, n=n, L=L) for s, n, L in
               ((41, 300, (7.0, 7.0, 7.5)), (42, 450, (8.0, 8.0, 8.0)), (43, 200, (6.0, 6.5, 7.0)))]
    pos = np.concatenate([x for x, _, _ in systems])
    vel = np.concatenate([v for _, v, _ in systems])
    kw = dict(sigma=SIG, cutoff=SIG, skin=SKIN, dt=0.001)
    with md.MDContext(pos, vel, [L for _, _, L in systems], counts=[x.shape[0] for x, _, _ in systems],
                      precision=md.MD_DW, rebuild_every=0, **kw) as ctx:
        ctx.set_spring_dashpot(300.0, 1.5)
        ctx.run(150)
        xg = ctx.positions()
        assert ctx.info().rebuilds > 1
    o = 0
    for x, v, L in systems:
        xr, _, _ = orc.vv_run(x, v, L, 150, potential=1, k_spring=300.0, gamma=1.5,
                              rebuild_every=0, **kw)
        d = np.mod(xg[o:o + x.shape[0]] - xr + L / 2, L) - L / 2
        assert np.abs(d).max() < 1e-9
        o += x.shape[0]
    k, g, u, dt = 1000.0, 5.0, 1.0, 1e-5
    zeta = g / (2.0 * math.sqrt(0.5 * k))
    e = math.exp(-zeta * math.pi / math.sqrt(1.0 - zeta ** 2))
    wd = math.sqrt(k / 0.5) * math.sqrt(1.0 - zeta ** 2)
    L = np.array([20.0, 20.0, 20.0])
    x = np.array([[10.0, 10.0, 10.0], [10.0 + SIG + 0.25 * u * dt, 10.0, 10.0]])
    v = np.array([[0.5 * u, 0.0, 0.0], [-0.5 * u, 0.0, 0.0]])
    with sd_ctx(md, x, v, L, k, g, precision=md.MD_DW, dt=dt) as ctx:
        ctx.run(int(1.5 * math.pi / wd / dt))
        vn = ctx.velocities()
    assert abs((vn[1, 0] - vn[0, 0]) / u - e) < 1e-4
    assert abs(vn[:, 0].sum()) < 1e-12
