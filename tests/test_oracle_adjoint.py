"""Pins of the oracle's FP64 trajectory gradient.

The reverse sweep (oracle/md_oracle_adjoint.c) is checked against central
finite differences of the oracle's own forward loss, which is written
separately and shares only the force/energy primitives pinned in
test_oracle_pins.py.  The pair Jacobian-vector product is checked against
finite differences of the forces.
"""
import numpy as np
import pytest

from paper_2009_07400_gb300 import inputs


@pytest.fixture(scope="module")
def small(orc):
    s = inputs.fcc_system(4, jitter=0.05, seed=41)        # 256 atoms
    x, v, _ = orc.vv_run(s.pos, s.vel, s.box, 40)
    return orc.wrap(x, s.box), v, s.box


def test_jvp_matches_force_differences(orc, small):
    x, _, L = small
    rng = np.random.default_rng(1)
    u = rng.normal(size=x.shape)
    h = 1e-6
    fd = (orc.forces_brute(x + h * u, L) - orc.forces_brute(x - h * u, L)) / (2 * h)
    ju = orc.jvp(x, u, L)
    assert np.abs(ju - fd).max() < 1e-6 * np.abs(fd).max()
    # J is symmetric: w . (J u) == u . (J w)
    w = rng.normal(size=x.shape)
    assert np.sum(w * ju) == pytest.approx(np.sum(u * orc.jvp(x, w, L)), rel=1e-11)


def directions(x0, gx, gv, seed):
    """Unit directions for directional derivatives: the gradients themselves,
    two random ones and two single coordinates, for x0 and for v0."""
    rng = np.random.default_rng(seed)
    out = [("x", gx / np.linalg.norm(gx)), ("v", gv / np.linalg.norm(gv))]
    for _ in range(2):
        u = rng.normal(size=x0.shape)
        u /= np.linalg.norm(u)
        out += [("x", u), ("v", u)]
    for a, c in ((7, 2), (100, 0)):
        u = np.zeros_like(x0)
        u[a % x0.shape[0], c] = 1.0
        out += [("x", u), ("v", u)]
    return out


def check_directional(g_u, fd, tol=1e-6):
    """g.u against finite differences, relative to the quantity itself.
    First the central quotient at h = 1e-6: |g.u - FD(1e-6)| <= tol |FD|.  A
    small g.u (|g.u| << |g|, e.g. single v0 coordinates, ~0.01-0.3 against
    |loss| ~ 3e3) can sit below the round-off floor of that quotient
    (~|loss| 1e-15 / h).  Then the fourth-order quotient from h = 1e-4 and
    2e-4 (Richardson: (4 FD(h) - FD(2h)) / 3, truncation O(h^4), round-off
    100x lower) must meet the same tol, and the miss at h = 1e-6 must lie
    within the floor the two estimates show, |FD(1e-6) - FD4|."""
    f6 = fd(1e-6)
    if abs(g_u - f6) <= tol * abs(f6):
        return "h=1e-6"
    f4 = (4.0 * fd(1e-4) - fd(2e-4)) / 3.0
    assert abs(g_u - f4) <= tol * abs(f4), (g_u, f6, f4)
    assert abs(g_u - f6) <= 1.5 * abs(f6 - f4) + tol * abs(f6), (g_u, f6, f4)
    return "4th order, h=1e-4"


@pytest.mark.parametrize("nsteps,window,every", [(30, 10, 20), (45, 15, 10)])
def test_adjoint_matches_finite_differences(orc, small, nsteps, window, every):
    """Central differences of the loss with the base run's lists and inside-rc
    pair sets frozen (the smooth branch the adjoint follows), each quantity
    judged relative to itself: dL/deps, dL/dsigma and directional derivatives
    along unit directions in x0 and v0 within 1e-6."""
    x0, v0, L = small
    kw = dict(rebuild_every=every)
    loss, ge, gs, gx, gv = orc.adjoint(x0, v0, L, nsteps, window, **kw)
    assert loss == pytest.approx(orc.traj_loss(x0, v0, L, nsteps, window, **kw), rel=1e-13)
    frozen = orc.FrozenLoss(x0, v0, L, nsteps, window, **kw)
    assert frozen.base == pytest.approx(loss, rel=1e-13)
    assert frozen(x0, v0) == pytest.approx(loss, rel=1e-13)
    h = 1e-6
    fd_e = (frozen(x0, v0, epsilon=1 + h) - frozen(x0, v0, epsilon=1 - h)) / (2 * h)
    fd_s = (frozen(x0, v0, sigma=1 + h) - frozen(x0, v0, sigma=1 - h)) / (2 * h)
    assert ge == pytest.approx(fd_e, rel=1e-6)
    assert gs == pytest.approx(fd_s, rel=1e-6)
    used = []
    for which, u in directions(x0, gx, gv, nsteps):
        g = gx if which == "x" else gv

        def fd(hh):
            if which == "x":
                return (frozen(x0 + hh * u, v0) - frozen(x0 - hh * u, v0)) / (2 * hh)
            return (frozen(x0, v0 + hh * u) - frozen(x0, v0 - hh * u)) / (2 * hh)
        used.append(check_directional(float(np.sum(g * u)), fd))
    # the gradient directions (largest g.u) always meet 1e-6 at h = 1e-6
    assert used[0] == "h=1e-6" and used[1] == "h=1e-6"


def test_adjoint_raw_fd_short(orc, small):
    """On a rollout short enough that no cutoff crossing moves, the raw loss
    is smooth and its plain central differences agree too."""
    x0, v0, L = small
    loss, ge, gs, _, _ = orc.adjoint(x0, v0, L, 5, 2)
    h = 1e-6
    for key, g in (("epsilon", ge), ("sigma", gs)):
        fd = (orc.traj_loss(x0, v0, L, 5, 2, **{key: 1 + h}) -
              orc.traj_loss(x0, v0, L, 5, 2, **{key: 1 - h})) / (2 * h)
        assert g == pytest.approx(fd, rel=1e-6)


def test_energy_gradient_homogeneity(orc, small):
    """Closed form: PE is linear in eps, so dLoss/deps == Loss/eps for a
    zero-step rollout window over the initial configuration only."""
    x0, v0, L = small
    loss, ge, _, _, _ = orc.adjoint(x0, v0, L, 1, 1, epsilon=1.7)
    # one step: x_1 depends on eps through F(x_0), so compare with FD instead
    h = 1e-6
    fd = (orc.traj_loss(x0, v0, L, 1, 1, epsilon=1.7 + h) -
          orc.traj_loss(x0, v0, L, 1, 1, epsilon=1.7 - h)) / (2 * h)
    assert ge == pytest.approx(fd, rel=1e-7)
    assert ge == pytest.approx(loss / 1.7, rel=1e-2)   # dominated by the direct term
