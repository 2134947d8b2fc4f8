"""Pins of the FP64 oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
a closed form of the 12-6 potential (Sec. 3.2, Eq. 2), textbook FCC lattice
geometry (tests/golden/fcc_shells.txt), brute force, conservation laws,
finite differences of the separately written energy, or an independent ODE
solver.  A dropped term, a wrong sign, a transposed index or a wrong power in
the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2009_07400_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RC, SKIN = 2.5, 0.3


def fcc_shells():
    rows = []
    with open(os.path.join(GOLDEN, "fcc_shells.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, z = line.split()
                rows.append((int(k), int(z)))
    return rows


def lattice_sums(density, eps=1.0, sigma=1.0, rc=RC):
    """PE per atom and pair virial per atom of a perfect FCC lattice, from the
    textbook shells: 1/2 sum_k z_k V(r_k), 1/2 sum_k z_k r_k F(r_k)."""
    a = (4.0 / density) ** (1.0 / 3.0)
    d1 = a / math.sqrt(2.0)
    pe = w = 0.0
    for k, z in fcc_shells():
        r = d1 * math.sqrt(k)
        if r < rc:
            v = 4 * eps * ((sigma / r) ** 12 - (sigma / r) ** 6)
            fmag = 24 * eps / r * (2 * (sigma / r) ** 12 - (sigma / r) ** 6)  # -dV/dr
            pe += 0.5 * z * v
            w += 0.5 * z * r * fmag
    return pe, w


def shell_count(density, r):
    a = (4.0 / density) ** (1.0 / 3.0)
    d1 = a / math.sqrt(2.0)
    return sum(z for k, z in fcc_shells() if d1 * math.sqrt(k) < r)


def dimer(r, L=20.0, axis=0):
    x = np.full((2, 3), 5.0)
    x[1, axis] += r
    return x, np.full(3, L)


# --------------------------------------------------------------------------
# Closed forms of the pair force and energy (Sec. 3.2, Eq. 2 and the commented
# potential beside it).
# --------------------------------------------------------------------------

@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (2.0, 1.3), (0.7, 0.9)])
def test_pair_closed_forms(orc, eps, sigma):
    rmin = 2 ** (1 / 6) * sigma
    x, L = dimer(rmin)
    F = orc.forces_brute(x, L, epsilon=eps, sigma=sigma)
    assert np.abs(F).max() < 1e-12 * 24 * eps / sigma          # force zero at the minimum
    pe, _ = orc.energy(x, L, epsilon=eps, sigma=sigma)
    assert pe == pytest.approx(-eps, rel=1e-13)                  # well depth eps
    x, L = dimer(sigma)
    F = orc.forces_brute(x, L, epsilon=eps, sigma=sigma)
    pe, w = orc.energy(x, L, epsilon=eps, sigma=sigma)
    assert abs(pe) < 1e-12 * eps                                 # V(sigma) = 0
    # |F(sigma)| = 24 eps / sigma, repulsive: atom 0 sits at lower x, pushed to -x
    assert F[0, 0] == pytest.approx(-24 * eps / sigma, rel=1e-13)
    assert F[1, 0] == pytest.approx(24 * eps / sigma, rel=1e-13)
    assert np.abs(F[:, 1:]).max() == 0.0
    # virial of one pair = r . F = r |F| (repulsive, positive)
    assert w == pytest.approx(sigma * 24 * eps / sigma, rel=1e-13)
    # attractive side
    x, L = dimer(1.5 * sigma, axis=2)
    F = orc.forces_brute(x, L, epsilon=eps, sigma=sigma)
    assert F[0, 2] > 0 and F[1, 2] < 0


def test_pair_force_general_r(orc):
    """|F(r)| = 24 eps (s/r)^6 [2 (s/r)^6 - 1] / r at several r (Eq. 2)."""
    eps, sigma = 1.7, 1.1
    for r in [0.95, 1.05, 1.3, 1.9, 2.4]:
        x, L = dimer(r, axis=1)
        F = orc.forces_brute(x, L, epsilon=eps, sigma=sigma)
        sr = sigma / r
        expect = 24 * eps * sr ** 6 * (2 * sr ** 6 - 1) / r
        assert F[1, 1] == pytest.approx(expect, rel=1e-13)


def test_strict_cutoff(orc):
    x, L = dimer(RC)
    assert np.abs(orc.forces_brute(x, L)).max() == 0.0
    assert orc.energy(x, L)[0] == 0.0
    x, L = dimer(RC - 1e-9)
    assert np.abs(orc.forces_brute(x, L)).max() > 0.0
    # the list radius is strict too
    x, L = dimer(RC + SKIN)
    assert [len(r) for r in orc.neighbors_brute(x, L, RC + SKIN)] == [0, 0]


def test_minimum_image_across_boundary(orc):
    """A pair split by the periodic boundary interacts through its image
    (periodic in every direction, Sec. 3.2)."""
    L = np.array([10.0, 11.0, 12.0])
    x = np.array([[0.2, 5.0, 5.0], [9.5, 5.0, 5.0]])      # image distance 0.7
    y = np.array([[0.2, 5.0, 5.0], [0.9, 5.0, 5.0]])      # direct distance 0.7
    Fx = orc.forces_brute(x, L)
    Fy = orc.forces_brute(y, L)
    assert Fx[0, 0] == pytest.approx(-Fy[0, 0], rel=1e-12)  # mirrored geometry
    assert abs(Fx[0, 0]) > 100


# --------------------------------------------------------------------------
# Forces are minus the gradient of the (separately written) potential energy.
# --------------------------------------------------------------------------

def test_force_is_minus_gradient(orc):
    s = inputs.fcc_system(4, jitter=0.12, seed=11)
    eps, sigma = 1.3, 0.95
    F = orc.forces_brute(s.pos, s.box, epsilon=eps, sigma=sigma)
    rng = np.random.default_rng(3)
    h = 1e-6
    for i in rng.choice(s.n, 6, replace=False):
        for d in range(3):
            xp = s.pos.copy()
            xm = s.pos.copy()
            xp[i, d] += h
            xm[i, d] -= h
            ep = orc.energy(xp, s.box, epsilon=eps, sigma=sigma)[0]
            em = orc.energy(xm, s.box, epsilon=eps, sigma=sigma)[0]
            fd = -(ep - em) / (2 * h)
            assert fd == pytest.approx(F[i, d], rel=1e-5, abs=1e-5)


# --------------------------------------------------------------------------
# Perfect FCC lattices: exact neighbour counts, zero forces, textbook energy.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n_cells,density", [(8, 0.8442), (7, 0.8442), (6, 0.9)])
def test_fcc_lattice(orc, n_cells, density):
    s = inputs.fcc_system(n_cells, density=density, jitter=0.0, seed=5)
    x = orc.wrap(s.pos, s.box)
    full = orc.neighbors_cells(x, s.box, RC + SKIN)
    half = orc.neighbors_cells(x, s.box, RC + SKIN, half=True)
    z_skin = shell_count(density, RC + SKIN)
    assert {len(r) for r in full} == {z_skin}
    assert sum(len(r) for r in half) * 2 == z_skin * s.n
    # half rows are balanced: each row holds about half of its neighbours
    assert max(len(r) for r in half) <= 0.75 * z_skin
    within_rc = orc.neighbors_cells(x, s.box, RC)
    assert {len(r) for r in within_rc} == {shell_count(density, RC)}
    pe_exact, w_exact = lattice_sums(density)
    pe, w = orc.energy_list(x, s.box, half, half=True)
    assert pe / s.n == pytest.approx(pe_exact, rel=1e-12)
    assert w / s.n == pytest.approx(w_exact, rel=1e-11)
    F = orc.forces_list(x, s.box, full)
    assert np.abs(F).max() < 1e-11
    if density == 0.8442:
        assert z_skin == 78 and shell_count(density, RC) == 54


# --------------------------------------------------------------------------
# Cell-list build == brute force (sets) on tiny boxes, incl. nc < 3.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("L,n,half", [
    ((5.7, 5.7, 5.7), 150, False),      # nc = 2: de-duplicated stencil
    ((5.7, 9.0, 12.0), 400, True),      # nc = (2, 3, 4), anisotropic
    ((9.0, 9.0, 9.0), 500, False),      # nc = 3
    ((12.0, 8.5, 11.3), 700, True),     # nc = (4, 3, 4)
    ((12.0, 12.0, 12.0), 900, False),   # nc = 4
])
def test_cells_equal_brute(orc, L, n, half):
    s = inputs.uniform_box(n, L, seed=n)
    x = orc.wrap(s.pos, s.box)
    a = orc.neighbors_brute(x, s.box, RC + SKIN, half=half)
    b = orc.neighbors_cells(x, s.box, RC + SKIN, half=half)
    for ra, rb in zip(a, b):
        assert len(set(rb.tolist())) == len(rb)          # no duplicates
        assert sorted(ra.tolist()) == sorted(rb.tolist())
    # a half list holds every pair of the full list exactly once
    if half:
        full = orc.neighbors_brute(x, s.box, RC + SKIN)
        pairs_full = {(min(i, j), max(i, j)) for i, r in enumerate(full) for j in r.tolist()}
        pairs_half = [(min(i, j), max(i, j)) for i, r in enumerate(b) for j in r.tolist()]
        assert len(pairs_half) == len(set(pairs_half)) == len(pairs_full)
        assert set(pairs_half) == pairs_full


def test_neighbors_sample_equals_full_rows(orc):
    """The sampled rows are the full cell-list rows of those atoms, in the
    same order (nc = 2 de-duplication included)."""
    for L, n in (((5.7, 5.7, 5.7), 150), ((12.0, 8.5, 11.3), 700)):
        s = inputs.uniform_box(n, L, seed=11)
        x = orc.wrap(s.pos, s.box)
        c_all, r_all = orc.neighbors_cells_raw(x, s.box, RC + SKIN)
        ids = np.random.default_rng(2).choice(n, 40, replace=False)
        c_s, r_s = orc.neighbors_sample(x, s.box, RC + SKIN, ids, cap=r_all.shape[1])
        assert np.array_equal(c_s, c_all[ids])
        for q, i in enumerate(ids):
            assert np.array_equal(r_s[q, :c_s[q]], r_all[i, :c_all[i]])


def test_binning(orc):
    L = np.array([9.0, 11.0, 13.0])
    s = inputs.uniform_box(600, L, seed=2)
    pos = s.pos.copy()
    pos[0] = [L[0] - 1e-15, 0.0, 4.5]        # next to the upper face
    pos[1] = [-1e-3, L[1] + 1e-3, 13.0]      # outside: wrapped
    x = orc.wrap(pos, L)
    assert np.all(x >= 0) and np.all(x <= L)
    assert x[1, 0] == pytest.approx(L[0] - 1e-3) and x[1, 1] == pytest.approx(1e-3)
    cell_of, start, atoms = orc.bin_cells(x, L, RC + SKIN)
    nc, cs = orc.cell_grid(L, RC + SKIN)
    assert list(nc) == [3, 3, 4]
    assert start[0] == 0 and start[-1] == s.n and np.all(np.diff(start) >= 0)
    for c in range(int(np.prod(nc))):
        members = atoms[start[c]:start[c + 1]]
        assert np.all(np.diff(members) > 0)               # stable: ascending ids
        assert np.all(cell_of[members] == c)
    # each atom is inside its cell (cell side s = L / nc)
    cx = cell_of // (nc[1] * nc[2])
    cy = (cell_of // nc[2]) % nc[1]
    cz = cell_of % nc[2]
    for d, c in enumerate([cx, cy, cz]):
        lo = c * cs[d]
        assert np.all(x[:, d] >= lo - 1e-12) and np.all(x[:, d] <= lo + cs[d] + 1e-12)


# --------------------------------------------------------------------------
# Invariants.
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def liquid(orc):
    """A disordered state: jittered FCC after 60 oracle steps at T = 1.44."""
    s = inputs.fcc_system(6, jitter=0.05, seed=21)
    x, v, _ = orc.vv_run(s.pos, s.vel, s.box, 60)
    return x, v, s.box


def test_newton_third_law(orc, liquid):
    x, _, L = liquid
    xw = orc.wrap(x, L)
    for half in (False, True):
        rows = orc.neighbors_cells(xw, L, RC + SKIN, half=half)
        F = orc.forces_list(xw, L, rows, half=half)
        assert np.abs(F.sum(axis=0)).max() < 1e-11 * np.abs(F).sum()


def test_full_half_brute_agree(orc, liquid):
    x, _, L = liquid
    xw = orc.wrap(x, L)
    Fb = orc.forces_brute(xw, L)
    for half in (False, True):
        rows = orc.neighbors_cells(xw, L, RC + SKIN, half=half)
        F = orc.forces_list(xw, L, rows, half=half)
        assert np.abs(F - Fb).max() < 1e-11 * np.abs(Fb).max()


def test_translation_and_permutation(orc, liquid):
    x, _, L = liquid
    F = orc.forces_brute(x, L)
    shift = np.array([0.37, -1.91, 4.2])
    Ft = orc.forces_brute(np.mod(x + shift, L), L)
    assert np.abs(Ft - F).max() < 1e-10 * np.abs(F).max()
    perm = np.random.default_rng(9).permutation(x.shape[0])
    Fp = orc.forces_brute(x[perm], L)
    assert np.abs(Fp - F[perm]).max() < 1e-11 * np.abs(F).max()


def test_forces_sample(orc, liquid):
    x, _, L = liquid
    ids = np.array([0, 5, 77, x.shape[0] - 1])
    Fs = orc.forces_sample(x, L, ids)
    Fb = orc.forces_brute(x, L)
    assert np.abs(Fs - Fb[ids]).max() < 1e-11 * np.abs(Fb).max()


def test_temperature_of_inputs():
    s = inputs.fcc_system(5, temperature=1.44, seed=3)
    t = np.sum(s.vel ** 2) / (3 * s.n - 3)
    assert t == pytest.approx(1.44, rel=1e-12)
    assert np.abs(s.vel.sum(axis=0)).max() < 1e-10


def test_thermo_closed_forms(orc):
    """orc_thermo against closed forms: with W = 0 it is the ideal-gas law
    P = rho T; with the inputs' velocities T is the 1.44 they were drawn at
    (3N - 3 degrees of freedom, momentum removed); a perfect FCC lattice at
    rest has T = 0 and P = W / (3V) with W the textbook shell sum; one atom
    has no free degree."""
    s = inputs.fcc_system(5, temperature=1.44, seed=3)
    vol = float(np.prod(s.box))
    th = orc.thermo(0.0, orc.kinetic(s.vel), 0.0, s.n, s.box)
    assert th["temperature"] == pytest.approx(1.44, rel=1e-12)
    assert th["pressure"] == pytest.approx(s.n / vol * 1.44, rel=1e-12)
    lat = inputs.fcc_system(5, density=0.8442, jitter=0.0, seed=5)
    x = orc.wrap(lat.pos, lat.box)
    pe, w = orc.energy_list(x, lat.box, orc.neighbors_cells(x, lat.box, RC + SKIN, half=True),
                            half=True)
    pe_exact, w_exact = lattice_sums(0.8442)
    th = orc.thermo(pe, 0.0, w, lat.n, lat.box)
    assert th["temperature"] == 0.0
    assert th["pressure"] == pytest.approx(0.8442 * w_exact / 3.0, rel=1e-10)
    assert th["etot"] == pytest.approx(lat.n * pe_exact, rel=1e-12)
    one = orc.thermo(-1.0, 2.0, 3.0, 1, 10.0)
    assert one["temperature"] == 0.0 and one["pressure"] == 0.0 and one["etot"] == 1.0


# --------------------------------------------------------------------------
# Velocity Verlet (Eq. 1): second order, time reversible, energy conserving.
# --------------------------------------------------------------------------

def dimer_exact(r0, vrel, t):
    """Relative coordinate of a LJ dimer (reduced mass 1/2) by an independent
    high-accuracy ODE solve."""
    from scipy.integrate import solve_ivp

    def rhs(_, y):
        r, u = y
        fmag = 24 * (2 * r ** -13 - r ** -7)       # -dV/dr, eps = sigma = 1
        return [u, fmag / 0.5]

    sol = solve_ivp(rhs, (0, t), [r0, vrel], rtol=1e-13, atol=1e-13, method="DOP853")
    return sol.y[0, -1]


def test_verlet_second_order(orc):
    r0, vrel, T = 1.4, -0.8, 1.0
    errs = []
    for dt in (0.01, 0.005, 0.0025):
        x, L = dimer(r0)
        v = np.zeros((2, 3))
        v[0, 0], v[1, 0] = -vrel / 2, vrel / 2
        nsteps = int(round(T / dt))
        xn, _, _ = orc.vv_run(x, v, L, nsteps, dt=dt, rebuild_every=10 ** 9)
        r = xn[1, 0] - xn[0, 0]
        errs.append(abs(r - dimer_exact(r0, vrel, T)))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.15)


def test_time_reversible(orc, liquid):
    """Velocity Verlet retraces its path when v is negated, to roundoff, as
    long as every list used is valid (rebuilt often enough)."""
    x0, v0, L = liquid
    for n, every in ((10, 20), (40, 5)):
        x1, v1, _ = orc.vv_run(x0, v0, L, n, rebuild_every=every)
        x2, v2, _ = orc.vv_run(x1, -v1, L, n, rebuild_every=every)
        d = np.mod(x2 - x0 + L / 2, L) - L / 2
        assert np.abs(d).max() < 1e-10
        assert np.abs(v2 + v0).max() < 1e-9


def test_fixed_schedule_can_go_stale(orc, liquid):
    """The fixed 20-step rebuild of Sec. 6 is a heuristic: at T = 1.44 the
    fastest atoms cross more than skin/2 in 20 steps, and forces over the
    old list then miss pairs.  Lists are exact while they are fresh."""
    x0, v0, L = liquid
    xw = orc.wrap(x0, L)
    rows = orc.neighbors_cells(xw, L, RC + SKIN)
    x5, _, _ = orc.vv_run(xw, v0, L, 5, rebuild_every=10 ** 9)
    assert np.abs(orc.forces_list(x5, L, rows) - orc.forces_brute(x5, L)).max() < 1e-10
    x19, _, _ = orc.vv_run(xw, v0, L, 19, rebuild_every=10 ** 9)
    disp = np.linalg.norm(x19 - xw, axis=1)
    stale = np.abs(orc.forces_list(x19, L, rows) - orc.forces_brute(x19, L)).max(axis=1) > 1e-10
    assert stale.sum() > 0 and disp.max() > SKIN / 2
    assert stale.sum() < 0.02 * x0.shape[0]


def test_displacement_schedule_keeps_lists_exact(orc, liquid):
    """With rebuild_every=0 (rebuild once an atom has moved more than skin/2
    since the last build) every list holds all pairs inside rc, so the run
    is the run with a fresh list at every step (rebuild_every=1), up to the
    summation order; the fixed 20-step schedule is not (its stale lists miss
    pairs at this temperature)."""
    x0, v0, L = liquid
    n = 100
    xa, va, Fa = orc.vv_run(x0, v0, L, n, rebuild_every=0)
    xb, vb, Fb = orc.vv_run(x0, v0, L, n, rebuild_every=1)
    xc, vc, _ = orc.vv_run(x0, v0, L, n, rebuild_every=20)
    mi = lambda d: np.mod(d + L / 2, L) - L / 2
    assert np.abs(mi(xa - xb)).max() < 1e-9 and np.abs(va - vb).max() < 1e-8
    assert np.abs(Fa - orc.forces_brute(orc.wrap(xa, L), L)).max() < 1e-9
    assert np.abs(mi(xc - xb)).max() > 1e3 * np.abs(mi(xa - xb)).max()


def test_displacement_trigger_step_is_exact(orc):
    """One atom drifting at constant speed 1 (dt 0.005, skin 0.3) from just
    inside the box face: it has moved 0.005 k after k steps, so the rule
    "rebuild once some atom moved more than skin/2" first fires at k = 31
    (0.155 > 0.15; at k = 30 the distance equals 0.15).  The rebuild wraps
    the coordinate back into the box, which makes the step visible."""
    L = np.array([20.0, 20.0, 20.0])
    x = np.array([[20.0 - 0.12, 10.0, 10.0], [5.0, 5.0, 5.0]])
    v = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    for k, wrapped in ((30, False), (31, True)):
        xk, _, _ = orc.vv_run(x, v, L, k, rebuild_every=0)
        assert (xk[0, 0] < L[0]) == wrapped, k
        assert abs(xk[0, 0] % L[0] - (20.0 - 0.12 + 0.005 * k) % L[0]) < 1e-12


def test_nve_energy(orc):
    """Total energy is conserved while KE and PE exchange; the residual comes
    from pairs crossing the unshifted cutoff, which no dt removes (the
    dimer test pins the dt^2 order of the integrator itself)."""
    s = inputs.fcc_system(6, jitter=0.05, seed=31)
    for dt, n in ((0.005, 200), (0.0025, 400)):
        _, _, _, E = orc.vv_run(s.pos, s.vel, s.box, n, dt=dt, energies=True)
        etot = E[:, 0] + E[:, 1]
        assert np.std(etot) < 0.02 * np.std(E[:, 1])
        drift = abs(etot[-n // 4:].mean() - etot[n // 4:n // 2].mean()) / s.n
        assert drift < 2e-4
