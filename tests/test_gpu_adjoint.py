"""Adjoint of the velocity-Verlet LJ rollout on the GPU vs the FP64 oracle.

Targets: FP64 path gradients within 1e-6 relative of central finite
differences (h = 1e-6) and of the FP64 oracle gradient.  Finite differences
are taken of the loss with the base run's lists and inside-rc pair sets
frozen (the oracle's FrozenLoss): the unshifted cutoff makes the raw loss
jump by V(rc)/W whenever a perturbation moves a cutoff crossing to another
step.  Every finite-difference quantity (dL/deps, dL/dsigma, directional
derivatives along unit directions) is judged relative to itself; where the
round-off floor of the h = 1e-6 quotient is above 1e-6 of a small
directional derivative, h = 1e-4 decides and the floor is shown by the two
quotients (see check_directional).

Mixed path: its forward trajectory carries FP32 rounding equivalent to a
perturbation of the positions of order 1e-7 sigma, and the gradient of a
200-step chaotic rollout moves by ~2e-5 (x0, v0) under such a perturbation
even in exact FP64 arithmetic; FP64 pair terms in the reverse sweep do not
change the mixed result (md_set_adjoint_precision).  The mixed gradients are
therefore judged against the FP64 oracle gradient within 1e-4 and within
five times that measured sensitivity (the control in the test).
"""
import numpy as np
import pytest

from paper_2009_07400_gb300 import inputs

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def small(orc):
    s = inputs.fcc_system(5, jitter=0.05, seed=41)        # 500 atoms
    x, v, _ = orc.vv_run(s.pos, s.vel, s.box, 40)
    return orc.wrap(x, s.box), v, s.box


def rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("nsteps,window,every,ckpt,lanes", [(40, 10, 20, 10, 1), (60, 25, 20, 20, 2),
                                                            (30, 30, 10, 5, 4), (40, 10, 20, 10, 4)])
def test_adjoint_matches_oracle(md, orc, small, nsteps, window, every, ckpt, lanes):
    """FP64 path; the pair kernel runs with the context's lanes per atom."""
    x0, v0, L = small
    loss_o, ge_o, gs_o, gx_o, gv_o = orc.adjoint(x0, v0, L, nsteps, window, rebuild_every=every)
    with md.MDContext(x0, v0, L, precision=md.MD_FP64, rebuild_every=every,
                      threads_per_atom=lanes) as ctx:
        loss, ge, gs, gx, gv = ctx.adjoint(nsteps, window, ckpt)
        # the context is left at the initial state
        assert np.array_equal(ctx.positions(), orc.wrap(x0, L))
    assert rel(loss, loss_o) < 1e-12
    assert rel(ge, ge_o) < 1e-9
    assert rel(gs, gs_o) < 1e-9
    assert np.linalg.norm(gx - gx_o) < 1e-9 * np.linalg.norm(gx_o)
    assert np.linalg.norm(gv - gv_o) < 1e-9 * np.linalg.norm(gv_o)


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


def test_adjoint_matches_finite_differences(md, orc, small):
    x0, v0, L = small
    nsteps, window = 40, 15
    with md.MDContext(x0, v0, L, precision=md.MD_FP64) as ctx:
        loss, ge, gs, gx, gv = ctx.adjoint(nsteps, window, 10)
    frozen = orc.FrozenLoss(x0, v0, L, nsteps, window)
    assert rel(loss, frozen.base) < 1e-12
    h = 1e-6
    fd_e = (frozen(x0, v0, epsilon=1 + h) - frozen(x0, v0, epsilon=1 - h)) / (2 * h)
    fd_s = (frozen(x0, v0, sigma=1 + h) - frozen(x0, v0, sigma=1 - h)) / (2 * h)
    assert rel(ge, fd_e) < 1e-6
    assert rel(gs, fd_s) < 1e-6
    rng = np.random.default_rng(3)
    dirs = [("x", gx / np.linalg.norm(gx)), ("v", gv / np.linalg.norm(gv))]
    for _ in range(2):
        u = rng.normal(size=x0.shape)
        u /= np.linalg.norm(u)
        dirs += [("x", u), ("v", u)]
    u = np.zeros_like(x0)
    u[7, 2] = 1.0
    dirs += [("x", u), ("v", u)]
    used = []
    for which, u in dirs:
        g = gx if which == "x" else gv

        def fd(hh):
            if which == "x":
                return (frozen(x0 + hh * u, v0) - frozen(x0 - hh * u, v0)) / (2 * hh)
            return (frozen(x0, v0 + hh * u) - frozen(x0, v0 - hh * u)) / (2 * hh)
        used.append(check_directional(float(np.sum(g * u)), fd))
    assert used[0] == "h=1e-6" and used[1] == "h=1e-6"


def test_adjoint_eps_sigma_parameters(md, orc, small):
    x0, v0, L = small
    kw = dict(epsilon=1.3, sigma=0.97)
    loss_o, ge_o, gs_o, gx_o, _ = orc.adjoint(x0, v0, L, 20, 10, **kw)
    with md.MDContext(x0, v0, L, precision=md.MD_FP64, **kw) as ctx:
        loss, ge, gs, gx, _ = ctx.adjoint(20, 10, 10)
        ctx.set_lj(1.0, 1.0)
        loss1, _, _, _, _ = ctx.adjoint(20, 10, 10)
    assert rel(loss, loss_o) < 1e-12 and rel(ge, ge_o) < 1e-9 and rel(gs, gs_o) < 1e-9
    assert np.linalg.norm(gx - gx_o) < 1e-9 * np.linalg.norm(gx_o)
    assert rel(loss1, orc.traj_loss(x0, v0, L, 20, 10)) < 1e-12


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_adjoint_mixed_lanes(md, orc, small, lanes):
    """Mixed path (FP32 pair terms) with 1, 2 and 4 lanes per atom against the
    FP64 oracle gradient of a short rollout."""
    x0, v0, L = small
    loss_o, ge_o, gs_o, gx_o, gv_o = orc.adjoint(x0, v0, L, 40, 10)
    with md.MDContext(x0, v0, L, precision=md.MD_MIXED, threads_per_atom=lanes) as ctx:
        loss, ge, gs, gx, gv = ctx.adjoint(40, 10, 10)
    assert rel(loss, loss_o) < 1e-6
    for g, go in ((ge, ge_o), (gs, gs_o)):
        assert rel(g, go) < 1e-4
    assert np.linalg.norm(gx - gx_o) < 1e-4 * np.linalg.norm(gx_o)
    assert np.linalg.norm(gv - gv_o) < 1e-4 * np.linalg.norm(gv_o)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_full_config(md, orc, precision):
    """16,384 atoms, 200 steps, loss = mean PE over the last 50 steps,
    checkpoints every 10 steps.  FP64: within 1e-6 of the FP64 oracle
    gradient (per scalar, and relative norm of the x0 and v0 gradients).
    Mixed: against the same oracle gradient within 1e-4 and within five
    times a control, the change of the exact (FP64 path) gradient when the
    initial positions move by uniform +-1e-7 sigma, the scale of the mixed
    path's FP32 rounding."""
    s = inputs.workload("fcc16_16384")
    loss_o, ge_o, gs_o, gx_o, gv_o = orc.adjoint(s.pos, s.vel, s.box, 200, 50)
    prec = md.MD_FP64 if precision == "fp64" else md.MD_MIXED
    with md.MDContext(s.pos, s.vel, s.box, precision=prec) as ctx:
        loss, ge, gs, gx, gv = ctx.adjoint(200, 50, 10)

    def errs(a, b):
        return np.array([rel(a[0], b[0]), rel(a[1], b[1]),
                         np.linalg.norm(a[2] - b[2]) / np.linalg.norm(b[2]),
                         np.linalg.norm(a[3] - b[3]) / np.linalg.norm(b[3])])
    e = errs((ge, gs, gx, gv), (ge_o, gs_o, gx_o, gv_o))
    if precision == "fp64":
        assert rel(loss, loss_o) < 1e-12
        assert np.all(e < 1e-6), e
        return
    assert rel(loss, loss_o) < 1e-6
    dp = np.random.default_rng(5).uniform(-1e-7, 1e-7, s.pos.shape)
    with md.MDContext(s.pos + dp, s.vel, s.box, precision=md.MD_FP64) as ctx:
        _, ge_p, gs_p, gx_p, gv_p = ctx.adjoint(200, 50, 10)
    control = errs((ge_p, gs_p, gx_p, gv_p), (ge_o, gs_o, gx_o, gv_o))
    print("mixed errors (eps, sigma, x0, v0):", e, "control:", control)
    assert np.all(e < 1e-4), e
    assert np.all(e <= 5.0 * control + 1e-9), (e, control)


def test_adjoint_precision_of_pair_terms(md, orc, small):
    """md_set_adjoint_precision: a mixed context with FP64 pair terms in the
    reverse sweep differentiates its own (mixed) trajectory; the result
    differs from the FP32-pair result by far less than both differ from the
    FP64 oracle's gradient, and an FP64 context is unchanged by the call."""
    x0, v0, L = small
    ref = orc.adjoint(x0, v0, L, 40, 10)
    with md.MDContext(x0, v0, L, precision=md.MD_MIXED) as ctx:
        m32 = ctx.adjoint(40, 10, 10)
        ctx.set_adjoint_precision(md.MD_FP64)
        m64 = ctx.adjoint(40, 10, 10)
    with md.MDContext(x0, v0, L, precision=md.MD_FP64) as ctx:
        ctx.set_adjoint_precision(md.MD_FP64)
        d64 = ctx.adjoint(40, 10, 10)
    assert m32[0] == m64[0]                       # same forward run
    for k in (3, 4):
        diff = np.linalg.norm(m32[k] - m64[k])
        assert diff <= np.linalg.norm(m32[k] - ref[k]) + np.linalg.norm(m64[k] - ref[k])
        assert np.linalg.norm(d64[k] - ref[k]) < 1e-9 * np.linalg.norm(ref[k])
    with pytest.raises(md.MDError):
        md.MDContext(x0, v0, L, precision=md.MD_MIXED).set_adjoint_precision(7)


def test_autograd_function(md, orc, small):
    """torch.autograd through the adjoint: d loss / d (eps, sigma, x0)."""
    torch = pytest.importorskip("torch")
    from paper_2009_07400_gb300.autodiff import rollout_loss
    x0, v0, L = small
    eps = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    xt = torch.tensor(x0, dtype=torch.float64, requires_grad=True)
    with md.MDContext(x0, v0, L, precision=md.MD_FP64) as ctx:
        loss = rollout_loss(ctx, eps, sig, xt, torch.tensor(v0), nsteps=20, window=10, ckpt_every=10)
        (2.0 * loss).backward()
    loss_o, ge_o, gs_o, gx_o, _ = orc.adjoint(x0, v0, L, 20, 10)
    assert rel(loss.item(), loss_o) < 1e-12
    assert rel(eps.grad.item(), 2 * ge_o) < 1e-9
    assert rel(sig.grad.item(), 2 * gs_o) < 1e-9
    assert np.linalg.norm(xt.grad.numpy() - 2 * gx_o) < 1e-9 * np.linalg.norm(2 * gx_o)


def test_autograd_function_device(md, orc, small):
    """The same through CUDA tensors: the state goes in and the gradients
    come out on the device (md_set_state_device / md_adjoint_device)."""
    torch = pytest.importorskip("torch")
    from paper_2009_07400_gb300.autodiff import rollout_loss
    x0, v0, L = small
    eps = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    xt = torch.tensor(x0, dtype=torch.float64, device="cuda", requires_grad=True)
    vt = torch.tensor(v0, dtype=torch.float64, device="cuda", requires_grad=True)
    with md.MDContext(x0, v0, L, precision=md.MD_FP64) as ctx:
        loss = rollout_loss(ctx, eps, sig, xt, vt, nsteps=20, window=10, ckpt_every=10)
        (3.0 * loss).backward()
    assert xt.grad.is_cuda and vt.grad.is_cuda
    loss_o, ge_o, gs_o, gx_o, gv_o = orc.adjoint(x0, v0, L, 20, 10)
    assert rel(loss.item(), loss_o) < 1e-12
    assert rel(eps.grad.item(), 3 * ge_o) < 1e-9
    assert rel(sig.grad.item(), 3 * gs_o) < 1e-9
    gx = xt.grad.cpu().numpy()
    gv = vt.grad.cpu().numpy()
    assert np.linalg.norm(gx - 3 * gx_o) < 1e-9 * np.linalg.norm(3 * gx_o)
    assert np.linalg.norm(gv - 3 * gv_o) < 1e-9 * np.linalg.norm(3 * gv_o)


def test_adjoint_workspace_reuse(md, small):
    """md_adjoint keeps its workspace between calls and grows it when a call
    needs more checkpoints or a longer block: calls of growing and shrinking
    sizes on one context give the same bits as fresh contexts."""
    x0, v0, L = small
    calls = [(20, 10, 10), (60, 20, 10), (40, 10, 20), (20, 5, 5)]

    def run(ctx, a):
        return ctx.adjoint(*a)

    with md.MDContext(x0, v0, L, precision=md.MD_MIXED) as ctx:
        reused = [run(ctx, a) for a in calls]
    for a, got in zip(calls, reused):
        with md.MDContext(x0, v0, L, precision=md.MD_MIXED) as ctx:
            ref = run(ctx, a)
        assert got[0] == ref[0] and got[1] == ref[1] and got[2] == ref[2]
        assert np.array_equal(got[3], ref[3]) and np.array_equal(got[4], ref[4])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_list_overflow_reruns(md, orc, precision):
    """A list that overflows during the forward sweep is found after the
    sweep, which reruns from step 0 with a larger list: loss and gradients
    bit for bit those of a context with room to spare (the capacity changes
    neither the rows nor their order).  A perfect FCC lattice has rows of
    exactly 78 (capacity 80); its sixth shell (2.909 sigma) lies just
    outside rc + skin, so once the atoms move the rows built at step 20
    outgrow it."""
    s = inputs.fcc_system(5, jitter=0.0, seed=43)         # 500 atoms, T 1.44
    x0, v0, L = s.pos, s.vel, s.box
    prec = md.MD_FP64 if precision == "fp64" else md.MD_MIXED
    with md.MDContext(x0, v0, L, precision=prec, rebuild_every=20) as ref:
        want = ref.adjoint(100, 20, 10)
    with md.MDContext(x0, v0, L, precision=prec, rebuild_every=20) as ctx:
        ctx.set_capacity(ctx.info().max_neighbors)
        cap0 = ctx.info().list_capacity
        got = ctx.adjoint(100, 20, 10)
        assert ctx.info().list_capacity > cap0          # the sweep overflowed and grew it
    assert got[0] == want[0] and got[1] == want[1] and got[2] == want[2]
    assert np.array_equal(got[3], want[3]) and np.array_equal(got[4], want[4])


def test_adjoint_with_split_cells(md, orc, small):
    """FP64 adjoint on a context whose build scans split cells (its checkpoint
    restores rebin by octant): the same loss and gradients as with whole
    cells, up to the summation order of the rows (round-off)."""
    x0, v0, L = small
    out = []
    for split in (0, 1):
        with md.MDContext(x0, v0, L, precision=md.MD_FP64, rebuild_every=20) as ctx:
            ctx.set_cell_split(split)
            out.append(ctx.adjoint(60, 20, 10))
    (l0, e0, s0, gx0, gv0), (l1, e1, s1, gx1, gv1) = out
    assert l1 == pytest.approx(l0, rel=1e-12)
    assert e1 == pytest.approx(e0, rel=1e-10) and s1 == pytest.approx(s0, rel=1e-10)
    assert np.linalg.norm(gx1 - gx0) <= 1e-9 * np.linalg.norm(gx0)
    assert np.linalg.norm(gv1 - gv0) <= 1e-9 * np.linalg.norm(gv0)
