"""Double-word path (precision MD_DW) vs the FP64 oracle, through the C ABI.

The pair arithmetic runs in unevaluated sums of two FP32 numbers (~48
significant bits): forces must meet the FP64 path's bar and a tighter one,
|dF_i| <= 1e-11 max(|F_i|, F_rms) per atom (the arithmetic's own error is
~1e-13 of the pair terms; the positions are represented to ~2^-46 absolute,
next to FP64's ~1e-14 at box coordinates), and trajectories, energies and
lists follow the FP64 oracle as the FP64 path does.
"""
import numpy as np
import pytest

from paper_2009_07400_gb300 import inputs

pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3
DW_TOL = 1e-11


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


def force_err(F, Fr):
    frms = np.sqrt(np.mean(np.sum(Fr ** 2, axis=1)))
    scale = np.maximum(np.linalg.norm(Fr, axis=1), frms)
    return np.max(np.linalg.norm(F - Fr, axis=1) / scale)


def sorted_rows(counts, rows):
    big = np.iinfo(np.int32).max
    width = max(1, int(counts.max()))
    out = np.full((counts.shape[0], width), big, np.int64)
    mask = np.arange(width)[None, :] < counts[:, None]
    out[mask] = rows[:, :width][mask]
    out.sort(axis=1)
    return out


def mi(d, L):
    return np.mod(d + L / 2, L) - L / 2


def liquid(orc, n_cells=7, steps=60, seed=3):
    s = inputs.fcc_system(n_cells, jitter=0.05, seed=seed)
    x, v, _ = orc.vv_run(s.pos, s.vel, s.box, steps)
    return inputs.System(x, v, s.box, seed)


def dw_ctx(md, s, **kw):
    return md.MDContext(s.pos, s.vel, s.box, precision=md.MD_DW, **kw)


@pytest.mark.parametrize("tpa", [1, 2, 4, 8])
@pytest.mark.parametrize("case", ["jitter7", "liquid", "ragged", "aniso"])
def test_dw_force_parity(md, orc, case, tpa):
    """Per-atom forces of the first evaluation, with whole and split cells
    (the order of a cell's entries changes the rounding, not the bar)."""
    if case == "jitter7":
        s = inputs.fcc_system(7, jitter=0.1, seed=8)
    elif case == "liquid":
        s = liquid(orc)
    elif case == "aniso":
        s = inputs.fcc_system(6, jitter=0.1, seed=21)
        s = inputs.System(s.pos * [1.0, 1.3, 0.8], s.vel, s.box * [1.0, 1.3, 0.8], 21)
    else:
        s = inputs.replica_system(2999, 0.82, 1.3, seed=12)
    xw = orc.wrap(s.pos, s.box)
    Fr = orc.forces_list(xw, s.box, orc.neighbors_cells(xw, s.box, RC + SKIN))
    for split in (0, 1):
        with dw_ctx(md, s, threads_per_atom=tpa) as ctx:
            ctx.set_cell_split(split)
            err = force_err(ctx.forces(), Fr)
            print(case, tpa, split, "max |dF| / max(|F|, F_rms):", err)
            assert err <= DW_TOL


def test_dw_force_params(md, orc):
    s = liquid(orc, n_cells=6)
    kw = dict(epsilon=1.7, sigma=0.93, cutoff=2.2, skin=0.4)
    xw = orc.wrap(s.pos, s.box)
    Fr = orc.forces_list(xw, s.box, orc.neighbors_cells(xw, s.box, 2.6), epsilon=1.7,
                         sigma=0.93, cutoff=2.2, skin=0.4)
    with dw_ctx(md, s, **kw) as ctx:
        assert force_err(ctx.forces(), Fr) <= DW_TOL
        # md_set_lj changes the double-word constants too
        ctx.set_lj(1.0, 1.0)
        Fr1 = orc.forces_list(xw, s.box, orc.neighbors_cells(xw, s.box, 2.6), epsilon=1.0,
                              sigma=1.0, cutoff=2.2, skin=0.4)
        assert force_err(ctx.forces(), Fr1) <= DW_TOL


def test_dw_lists_and_energy(md, orc):
    """Lists (built from the high parts of the split positions) equal the
    oracle's rows; PE, KE and W at the FP64 path's tolerances."""
    s = liquid(orc)
    xw = orc.wrap(s.pos, s.box)
    pe, w = orc.energy_list(xw, s.box, orc.neighbors_cells(xw, s.box, RC + SKIN, half=True),
                            half=True)
    ke = orc.kinetic(s.vel)
    with dw_ctx(md, s) as ctx:
        c_g, r_g = ctx.neighbors_raw()
        c_o, r_o = orc.neighbors_cells_raw(xw, s.box, RC + SKIN)
        assert np.array_equal(c_g, c_o)
        assert np.array_equal(sorted_rows(c_g, r_g), sorted_rows(c_o, r_o))
        gpe, gke, gw = ctx.energy()
        assert gpe[0] == pytest.approx(pe, rel=1e-12)
        assert gke[0] == pytest.approx(ke, rel=1e-13)
        assert gw[0] == pytest.approx(w, rel=1e-11)


@pytest.mark.parametrize("tpa", [1, 4])
def test_dw_run_matches_oracle(md, orc, tpa):
    """100 steps of the 2,048-atom FCC workload (rebuild every 20): the FP64
    path's trajectory bar."""
    s = inputs.workload("fcc8_2048")
    x_ref, v_ref, _, E_ref = orc.vv_run(s.pos, s.vel, s.box, 100, energies=True)
    with dw_ctx(md, s, threads_per_atom=tpa) as ctx:
        E = ctx.run(100, energy_every=20)
        assert np.abs(mi(ctx.positions() - x_ref, s.box)).max() < 1e-9
        assert np.abs(ctx.velocities() - v_ref).max() < 1e-8
        for k in range(5):
            pe, ke, w = E[k, 0]
            assert pe == pytest.approx(E_ref[20 * k + 19, 0], rel=1e-10)
            assert ke == pytest.approx(E_ref[20 * k + 19, 1], rel=1e-10)
            assert w == pytest.approx(E_ref[20 * k + 19, 2], rel=1e-9)


def test_dw_chunks_equal_one_run(md, orc):
    """A run split into calls (graphs of other shapes) is bitwise the same."""
    s = liquid(orc, n_cells=6)
    with dw_ctx(md, s) as a, dw_ctx(md, s) as b:
        a.run(57)
        b.run(13)
        b.run(20)
        b.run(24)
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.velocities(), b.velocities())


def test_dw_131k_energy(md, orc):
    """The paper's CPU workload size (131,072 atoms): total energy after 100
    steps within 1e-10 relative of the oracle, as the FP64 path."""
    s = inputs.workload("fcc32_131072")
    x_ref, v_ref, _ = orc.vv_run(s.pos, s.vel, s.box, 100)
    e_ref = orc.energy(x_ref, s.box)[0] + orc.kinetic(v_ref)
    with dw_ctx(md, s) as ctx:
        E = ctx.run(100, energy_every=100)
    assert E[-1, 0, 0] + E[-1, 0, 1] == pytest.approx(e_ref, rel=1e-10)


def test_dw_full_size(md, orc):
    """1,048,576 atoms after a graph-replayed rebuild cycle: rows equal the
    oracle's, forces of 4,096 sampled atoms within the bar."""
    s = inputs.workload("fcc64_1048576")
    with dw_ctx(md, s) as ctx:
        ctx.run(20)
        x = ctx.positions()
        c_g, r_g = ctx.neighbors_raw()
        c_o, r_o = orc.neighbors_cells_raw(orc.wrap(x, s.box), s.box, RC + SKIN)
        assert np.array_equal(c_g, c_o)
        assert np.array_equal(sorted_rows(c_g, r_g), sorted_rows(c_o, r_o))
        ids = np.random.default_rng(0).choice(s.n, 4096, replace=False)
        Fr = orc.forces_sample(x, s.box, ids)
        assert force_err(ctx.forces()[ids], Fr) <= DW_TOL


def test_dw_batched_replicas(md, orc):
    reps = inputs.replica_ensemble(6, seed=77, n_min=500, n_max=3000)
    pos = np.concatenate([r.pos for r in reps])
    vel = np.concatenate([r.vel for r in reps])
    counts = [r.n for r in reps]
    with md.MDContext(pos, vel, [r.box for r in reps], counts=counts, precision=md.MD_DW) as ctx:
        F = ctx.forces()
        o = 0
        for r in reps:
            xw = orc.wrap(r.pos, r.box)
            Fr = orc.forces_list(xw, r.box, orc.neighbors_cells(xw, r.box, RC + SKIN))
            assert force_err(F[o:o + r.n], Fr) <= DW_TOL
            o += r.n
        E = ctx.run(40, energy_every=40)
        X = ctx.positions()
        o = 0
        for k, r in enumerate(reps):
            x_ref, _, _, E_ref = orc.vv_run(r.pos, r.vel, r.box, 40, energies=True)
            assert np.abs(mi(X[o:o + r.n] - x_ref, r.box)).max() < 1e-9
            assert E[0, k, 0] == pytest.approx(E_ref[-1, 0], rel=1e-10)
            o += r.n


def test_dw_displacement_trigger(md, orc):
    """rebuild_every = 0 on the double-word path follows the oracle's
    fresh-list run (the trigger reads the high parts of the positions)."""
    s = inputs.workload("fcc8_2048")
    x_ref, v_ref, F_ref = orc.vv_run(s.pos, s.vel, s.box, 200, rebuild_every=1)
    with dw_ctx(md, s, rebuild_every=0) as ctx:
        ctx.run(200)
        assert np.abs(mi(ctx.positions() - x_ref, s.box)).max() < 1e-9
        assert np.abs(ctx.velocities() - v_ref).max() < 1e-8
        assert force_err(ctx.forces(), F_ref) <= 1e-10


def test_dw_autotune(md, orc):
    """The autotuner tries full lists with 1, 2, 4 and 8 lanes and keeps the state."""
    s = liquid(orc, n_cells=6)
    with dw_ctx(md, s) as ctx:
        x0 = ctx.positions()
        chosen = ctx.autotune(20)
        assert chosen.list_type == md.MD_LIST_FULL
        assert chosen.threads_per_atom in (1, 2, 4, 8)
        assert np.array_equal(ctx.positions(), x0)


def test_dw_refusals(md, orc):
    """What the double-word path does not run is refused with MD_ERR_INVAL."""
    s = inputs.fcc_system(5, jitter=0.05, seed=4)
    for lt in (md.MD_LIST_HALF, md.MD_LIST_GROUP2, md.MD_LIST_GROUP4):
        with pytest.raises(md.MDError) as e:
            dw_ctx(md, s, list_type=lt)
        assert e.value.code == -1
    with dw_ctx(md, s) as ctx:
        with pytest.raises(md.MDError) as e:
            ctx.study_force_variant(0, 1)
        assert e.value.code in (-1, -9)
        ctx.run(10)                      # the context still runs


def test_dw_range_guard(md, orc):
    """An atom that runs more than a cell side beyond its cell between
    binnings (no interactions: a dilute lattice, one fast atom, binning only
    at the start) stops the double-word run with MD_ERR_BADPOS instead of
    losing the exactness of its split position; the other paths run on."""
    L = np.full(3, 30.0)                             # 10 cells of side 3 per edge
    g = (np.arange(4) * 7.5 + 1.0)
    pos = np.array([[a, b, c] for a in g for b in g for c in g])
    pos = np.concatenate([pos, [[2.0, 4.75, 4.75]]])   # 5.3 from every lattice line
    vel = np.zeros_like(pos)
    vel[-1] = [20.0, 0.0, 0.0]
    kw = dict(rebuild_every=100000)
    with md.MDContext(pos, vel, L, precision=md.MD_DW, **kw) as ctx:
        ctx.run(20)                                  # 2 units: still in range
        with pytest.raises(md.MDError) as e:
            ctx.run(200)
        assert e.value.code == -8
        assert "double-word" in str(e.value)
    for prec in (md.MD_FP64, md.MD_MIXED):
        with md.MDContext(pos, vel, L, precision=prec, **kw) as ctx:
            ctx.run(220)
            assert ctx.positions()[-1, 0] == pytest.approx(2.0 + 220 * 0.005 * 20.0, rel=1e-12)


def rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("pair", ["dw", "fp64"])
@pytest.mark.parametrize("nsteps,window,every,ckpt,lanes", [(40, 10, 20, 10, 1), (60, 25, 20, 20, 2),
                                                            (30, 30, 10, 5, 4)])
def test_dw_adjoint_matches_oracle(md, orc, nsteps, window, every, ckpt, lanes, pair):
    """md_adjoint on a double-word context (double-word forward and
    recompute; reverse pair terms in double word, the default, or in FP64)
    against the oracle's FP64 reverse sweep: the loss and every gradient far
    inside the FP64 path's bar."""
    s = inputs.fcc_system(5, jitter=0.05, seed=41)        # 500 atoms
    x, v, _ = orc.vv_run(s.pos, s.vel, s.box, 40)
    x0, v0, L = orc.wrap(x, s.box), v, s.box
    loss_o, ge_o, gs_o, gx_o, gv_o = orc.adjoint(x0, v0, L, nsteps, window, rebuild_every=every)
    with md.MDContext(x0, v0, L, precision=md.MD_DW, rebuild_every=every,
                      threads_per_atom=lanes) as ctx:
        if pair == "fp64":
            ctx.set_adjoint_precision(md.MD_FP64)
        loss, ge, gs, gx, gv = ctx.adjoint(nsteps, window, ckpt)
        again = ctx.adjoint(nsteps, window, ckpt)          # the workspace is reused
        xa = ctx.positions()
    e = [rel(loss, loss_o), rel(ge, ge_o), rel(gs, gs_o),
         np.linalg.norm(gx - gx_o) / np.linalg.norm(gx_o),
         np.linalg.norm(gv - gv_o) / np.linalg.norm(gv_o)]
    print(f"double-word adjoint, {pair} pair terms, errors (loss, eps, sigma, x0, v0):", e)
    assert e[0] < 1e-11 and max(e[1:]) < 1e-8
    assert again[0] == loss and np.array_equal(again[3], gx)
    assert np.array_equal(xa, x0) or np.abs(mi(xa - x0, L)).max() == 0.0


def test_dw_adjoint_full_config(md, orc):
    """16,384 atoms, 200 steps, window 50, checkpoints every 10, double-word
    pair terms: the FP64 path's bar (1e-6 per scalar and in relative norm)."""
    s = inputs.workload("fcc16_16384")
    loss_o, ge_o, gs_o, gx_o, gv_o = orc.adjoint(s.pos, s.vel, s.box, 200, 50)
    with dw_ctx(md, s) as ctx:
        loss, ge, gs, gx, gv = ctx.adjoint(200, 50, 10)
    e = [rel(loss, loss_o), rel(ge, ge_o), rel(gs, gs_o),
         np.linalg.norm(gx - gx_o) / np.linalg.norm(gx_o),
         np.linalg.norm(gv - gv_o) / np.linalg.norm(gv_o)]
    print("double-word adjoint, full config (loss, eps, sigma, x0, v0):", e)
    assert e[0] < 1e-12 and max(e[1:]) < 1e-6


def test_dw_adjoint_precision_refusals(md, orc):
    """MD_DW pair terms need a double-word context (split positions)."""
    s = inputs.fcc_system(4, jitter=0.05, seed=2)
    for prec in (md.MD_FP64, md.MD_MIXED):
        with md.MDContext(s.pos, s.vel, s.box, precision=prec) as ctx:
            with pytest.raises(md.MDError) as e:
                ctx.set_adjoint_precision(md.MD_DW)
            assert e.value.code == -1
    with dw_ctx(md, s) as ctx:
        for p in (md.MD_DW, md.MD_FP64, md.MD_MIXED):
            ctx.set_adjoint_precision(p)
        with pytest.raises(md.MDError):
            ctx.set_adjoint_precision(5)


def test_dw_nve_vs_oracle(md, orc):
    """1000 steps of the 131,072-atom FCC workload (rebuild every 20) against
    the FP64 oracle's run from the same state: the double-word path's force
    error (~1e-12) perturbs the trajectory far less than the FP32 scale that
    decorrelates the mixed path, so the literal total-energy criterion holds
    at every 100th step with room to spare (|dE| / N <= 1e-6; FP64 runs from
    states 1e-12 sigma apart differ by ~1e-7 per atom after 1000 steps).
    Measured on GB300: at most 2e-12 per atom up to step 800, then 1.2e-7,
    which is one pair crossing rc a step earlier or later than in the oracle's
    run (|V(rc)| / N = 1.24e-7 with the unshifted potential)."""
    s = inputs.workload("fcc32_131072")
    x_ref, v_ref, _, E_ref = orc.vv_run(s.pos, s.vel, s.box, 1000, energies=True)
    e_ref = E_ref[99::100, 0] + E_ref[99::100, 1]
    with dw_ctx(md, s) as ctx:
        E = ctx.run(1000, energy_every=100)
    de = (E[:, 0, 0] + E[:, 0, 1] - e_ref) / s.n
    print("double-word |dE|/N every 100 steps:", np.array2string(np.abs(de), precision=2))
    assert np.all(np.abs(de) <= 1e-6)


def test_dw_adjoint_mixed_pair_terms(md, orc):
    """A double-word context may also take FP32 pair terms in the reverse
    sweep (md_set_adjoint_precision(MD_MIXED)): the mixed path's bar."""
    s = inputs.fcc_system(5, jitter=0.05, seed=41)
    x, v, _ = orc.vv_run(s.pos, s.vel, s.box, 40)
    x0, v0, L = orc.wrap(x, s.box), v, s.box
    loss_o, ge_o, gs_o, gx_o, gv_o = orc.adjoint(x0, v0, L, 40, 10)
    with md.MDContext(x0, v0, L, precision=md.MD_DW) as ctx:
        ctx.set_adjoint_precision(md.MD_MIXED)
        loss, ge, gs, gx, gv = ctx.adjoint(40, 10, 10)
    assert rel(loss, loss_o) < 1e-11
    assert rel(ge, ge_o) < 1e-4 and rel(gs, gs_o) < 1e-4
    assert np.linalg.norm(gx - gx_o) < 1e-4 * np.linalg.norm(gx_o)
    assert np.linalg.norm(gv - gv_o) < 1e-4 * np.linalg.norm(gv_o)


@pytest.mark.parametrize("case", ["band", "band_wide", "edges", "s_eq_rs", "nc2"])
def test_dw_list_parity_edges(md, orc, case):
    """The double-word context's list build reads the high parts of the split
    positions (rounded to the replica's grid, not to FP32): rows still equal
    the oracle's on pairs within 1e-15 .. 1e-5 of the list radius, on
    coordinates at cell faces, mid-planes and box edges, with cells of side
    exactly rc + skin and with two cells per edge; whole and split cells."""
    import test_gpu_parity as tp
    if case == "band":
        s = tp.band_system()
    elif case == "band_wide":
        s = tp.band_system(seed=6, L=(8.39, 5.75, 30.0))
    elif case == "edges":
        s = tp.edge_coordinates()
    elif case == "s_eq_rs":
        s = inputs.uniform_box(1500, (5.6, 8.4, 11.2), seed=13)
    else:
        s = inputs.uniform_box(400, (5.7, 5.7, 5.7), seed=9)
    c_o, r_o = orc.neighbors_cells_raw(orc.wrap(s.pos, s.box), s.box, RC + SKIN)
    with dw_ctx(md, s) as ctx:
        for split in (1, 0):
            ctx.set_cell_split(split)
            c_g, r_g = ctx.neighbors_raw()
            assert np.array_equal(c_g, c_o)
            assert np.array_equal(sorted_rows(c_g, r_g), sorted_rows(c_o, r_o))


def test_dw_random_geometry_sweep(md, orc):
    """Twenty seeded random systems (1 to 6 cells per edge, anisotropic cells,
    so the grid step follows the largest cell side; densities 0.05 to 1.1;
    cutoff and skin varied): bit-exact lists and forces within the FP64
    path's bar of the plain definition (measured worst 4.7e-11: uniform
    random atoms include close pairs whose large forces nearly cancel)."""
    rng = np.random.default_rng(2025)
    worst = 0.0
    for case in range(20):
        rc = float(rng.uniform(1.2, 3.0))
        skin = float(rng.uniform(0.0, 0.6))
        rs = rc + skin
        L = rng.uniform(2.0, 6.5, 3) * rs
        rho = float(rng.uniform(0.05, 1.1))
        n = max(2, min(6000, int(rho * np.prod(L))))
        x = rng.uniform(0, 1, (n, 3)) * L
        v = rng.normal(size=(n, 3))
        with md.MDContext(x, v, L, precision=md.MD_DW, cutoff=rc, skin=skin) as ctx:
            c_g, r_g = ctx.neighbors_raw()
            c_o, r_o = orc.neighbors_cells_raw(orc.wrap(x, L), L, rs, cap=1024)
            assert np.array_equal(c_g, c_o), case
            assert np.array_equal(sorted_rows(c_g, r_g), sorted_rows(c_o, r_o)), case
            Fr = orc.forces_brute(x, L, cutoff=rc)
            err = force_err(ctx.forces(), Fr)
            worst = max(worst, err)
            assert err <= 1e-10, case
    print("double-word random geometries, worst force error:", worst)


def test_dw_autograd_function_device(md, orc):
    """torch.autograd through the adjoint of a double-word context with CUDA
    tensors in and out: loss and gradients at the FP64 path's bar."""
    torch = pytest.importorskip("torch")
    from paper_2009_07400_gb300.autodiff import rollout_loss
    s = inputs.fcc_system(5, jitter=0.05, seed=41)
    x, v, _ = orc.vv_run(s.pos, s.vel, s.box, 40)
    x0, v0, L = orc.wrap(x, s.box), v, s.box
    eps = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    xt = torch.tensor(x0, dtype=torch.float64, device="cuda", requires_grad=True)
    vt = torch.tensor(v0, dtype=torch.float64, device="cuda", requires_grad=True)
    with md.MDContext(x0, v0, L, precision=md.MD_DW) as ctx:
        loss = rollout_loss(ctx, eps, sig, xt, vt, nsteps=20, window=10, ckpt_every=10)
        (3.0 * loss).backward()
    assert xt.grad.is_cuda and vt.grad.is_cuda
    loss_o, ge_o, gs_o, gx_o, gv_o = orc.adjoint(x0, v0, L, 20, 10)
    assert rel(loss.item(), loss_o) < 1e-11
    assert rel(eps.grad.item(), 3 * ge_o) < 1e-9
    assert rel(sig.grad.item(), 3 * gs_o) < 1e-9
    gx = xt.grad.cpu().numpy()
    gv = vt.grad.cpu().numpy()
    assert np.linalg.norm(gx - 3 * gx_o) < 1e-9 * np.linalg.norm(3 * gx_o)
    assert np.linalg.norm(gv - 3 * gv_o) < 1e-9 * np.linalg.norm(3 * gv_o)
