"""The oracle's spring-dashpot contact model (Sec. 3.2, Eq. 3) pinned against
the closed-form damped collision of two spheres, the plain all-pairs
definition, Newton's third law and energy balance."""
import math

import numpy as np
import pytest

from paper_2009_07400_gb300 import inputs

SIG = 1.0


def _kw(k, g, dt=0.005, **extra):
    return dict(potential=1, k_spring=k, gamma=g, sigma=SIG, cutoff=SIG, skin=0.3, dt=dt,
                mass=1.0, **extra)


def _collide(orc, k, g, u, dt, steps):
    """Two spheres approaching head-on along x with relative speed u, from
    just outside contact; returns the relative velocity after `steps`."""
    L = np.array([20.0, 20.0, 20.0])
    x = np.array([[10.0, 10.0, 10.0], [10.0 + SIG + 0.25 * u * dt, 10.0, 10.0]])
    v = np.array([[0.5 * u, 0.0, 0.0], [-0.5 * u, 0.0, 0.0]])
    xn, vn, _ = orc.vv_run(x, v, L, steps, **_kw(k, g, dt=dt, rebuild_every=10 ** 9))
    return xn, vn, v


def test_restitution_matches_damped_oscillator(orc):
    """Overlap delta obeys delta'' + (gamma/mu) delta' + (K/mu) delta = 0 with
    mu = m/2 while in contact, so the pair leaves with relative speed
    e u, e = exp(-zeta pi / sqrt(1 - zeta^2)), zeta = gamma / (2 sqrt(mu K)),
    after a contact of pi / omega_d."""
    k, g, u = 1000.0, 5.0, 1.0
    mu = 0.5
    zeta = g / (2.0 * math.sqrt(mu * k))
    e = math.exp(-zeta * math.pi / math.sqrt(1.0 - zeta ** 2))
    wd = math.sqrt(k / mu) * math.sqrt(1.0 - zeta ** 2)
    dt = 1e-5
    steps = int(1.5 * math.pi / wd / dt)
    xn, vn, v0 = _collide(orc, k, g, u, dt, steps)
    rel = vn[1, 0] - vn[0, 0]
    assert rel > 0                                             # separating
    assert abs(rel / u - e) < 1e-4
    assert np.abs(vn.sum(axis=0) - v0.sum(axis=0)).max() < 1e-12   # momentum
    assert np.abs(vn[:, 1:]).max() == 0.0


def test_elastic_collision_conserves_energy(orc):
    """gamma = 0: the spheres leave with the approach speed (e = 1, up to the
    integrator's O(dt^2) error) and KE + 1/2 K delta^2 stays constant through
    the contact."""
    k, u = 1000.0, 1.0
    dt = 1e-5
    wd = math.sqrt(k / 0.5)
    steps = int(0.5 * math.pi / wd / dt)                       # mid-contact
    xm, vm, _ = _collide(orc, k, 0.0, u, dt, steps)
    delta = SIG - (xm[1, 0] - xm[0, 0])
    assert delta > 0
    e_mid = 0.5 * np.sum(vm ** 2) + 0.5 * k * delta ** 2
    e0 = 0.5 * (2 * (0.5 * u) ** 2)
    assert abs(e_mid - e0) / e0 < 1e-4
    xn, vn, _ = _collide(orc, k, 0.0, u, dt, 3 * steps)
    assert abs((vn[1, 0] - vn[0, 0]) / u - 1.0) < 1e-4


def _dense(seed=3, n=600):
    """Overlapping spheres (packing fraction ~0.75) with random velocities."""
    rng = np.random.default_rng(seed)
    L = np.array([8.0, 8.5, 9.0])
    x = rng.uniform(0, 1, (n, 3)) * L
    v = rng.normal(size=(n, 3))
    return x, v, L


def test_list_equals_plain_definition_and_third_law(orc):
    x, v, L = _dense()
    kw = _kw(500.0, 3.0)
    rows = orc.neighbors_cells(orc.wrap(x, L), L, SIG + 0.3)
    F = orc.forces_sd_list(orc.wrap(x, L), v, L, rows, **{k: kw[k] for k in ("k_spring", "gamma", "sigma")})
    Fb = orc.forces_sd_brute(x, v, L, **{k: kw[k] for k in ("k_spring", "gamma", "sigma")})
    assert np.abs(F - Fb).max() < 1e-12 * np.abs(Fb).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-10 * np.abs(F).sum()
    # the paper's static setting K = gamma = 0 exerts no force at all
    F0 = orc.forces_sd_brute(x, v, L, k_spring=0.0, gamma=0.0, sigma=SIG)
    assert np.all(F0 == 0.0)


def test_pair_force_direction_and_magnitude(orc):
    """One overlapping pair at rest: |F| = K (sigma - r), repulsive; moving
    apart along the line of centres adds -gamma v_n."""
    L = np.array([10.0, 10.0, 10.0])
    r = 0.9
    d = np.array([0.3, -0.4, 0.5]) / np.linalg.norm([0.3, -0.4, 0.5])
    x = np.array([[5.0, 5.0, 5.0], 5.0 + r * d])
    v = np.zeros((2, 3))
    F = orc.forces_sd_brute(x, v, L, k_spring=100.0, gamma=7.0, sigma=SIG)
    np.testing.assert_allclose(F[0], -100.0 * (SIG - r) * d, rtol=1e-13)
    np.testing.assert_allclose(F[1], 100.0 * (SIG - r) * d, rtol=1e-13)
    v[1] = 0.2 * d                                  # separating at 0.2
    F = orc.forces_sd_brute(x, v, L, k_spring=100.0, gamma=7.0, sigma=SIG)
    # x_01 . v_01 / r = (-d) . (-0.2 d) = 0.2 -> dashpot -gamma * 0.2 along xhat_01 = -d
    np.testing.assert_allclose(F[0], -(100.0 * (SIG - r) - 7.0 * 0.2) * d, rtol=1e-13)


def test_granular_gas_cools(orc):
    """With gamma > 0 a periodic gas of overlapping spheres loses energy:
    KE + elastic PE falls over the run, and with gamma = 0 it is conserved
    to the integrator's accuracy."""
    x, v, L = _dense(seed=9, n=400)
    x = orc.wrap(x, L)
    for g in (0.0, 2.0):
        kw = _kw(200.0, g, dt=0.001, rebuild_every=0)
        _, _, _, E = orc.vv_run(x, v, L, 400, energies=True, **kw)
        etot = E[:, 0] + E[:, 1]
        if g == 0.0:
            assert abs(etot[-1] - etot[0]) / abs(etot[0]) < 2e-3
        else:
            assert etot[-1] < 0.8 * etot[0]
            assert np.all(np.diff(etot[::20]) < 1e-6 * abs(etot[0]))
