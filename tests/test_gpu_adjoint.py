"""Adjoint of the velocity-Verlet LJ rollout on the GPU vs the FP64 oracle.

Targets: gradients within 1e-6 relative of central finite differences
(h = 1e-6) and of the FP64 oracle gradient.  Finite differences are taken
of the loss with the base run's lists and inside-rc pair sets frozen (the
oracle's FrozenLoss): the unshifted cutoff makes the raw loss jump by
V(rc)/W whenever a perturbation moves a cutoff crossing to another step.
Directional derivatives along unit vectors are judged normwise.
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
    for _ in range(2):
        u = rng.normal(size=x0.shape)
        u /= np.linalg.norm(u)
        fd_x = (frozen(x0 + h * u, v0) - frozen(x0 - h * u, v0)) / (2 * h)
        assert abs(np.sum(gx * u) - fd_x) <= 1e-6 * np.linalg.norm(gx)
        fd_v = (frozen(x0, v0 + h * u) - frozen(x0, v0 - h * u)) / (2 * h)
        assert abs(np.sum(gv * u) - fd_v) <= 1e-6 * np.linalg.norm(gv)


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
    gradient.  Mixed: compared with the same FP64 oracle gradient; its error
    comes from the FP32 pair arithmetic amplified along the chaotic rollout."""
    s = inputs.workload("fcc16_16384")
    loss_o, ge_o, gs_o, gx_o, gv_o = orc.adjoint(s.pos, s.vel, s.box, 200, 50)
    prec = md.MD_FP64 if precision == "fp64" else md.MD_MIXED
    with md.MDContext(s.pos, s.vel, s.box, precision=prec) as ctx:
        loss, ge, gs, gx, gv = ctx.adjoint(200, 50, 10)
    tol = 1e-6 if precision == "fp64" else 1e-3
    assert rel(loss, loss_o) < (1e-12 if precision == "fp64" else 1e-5)
    assert rel(ge, ge_o) < tol
    assert rel(gs, gs_o) < tol
    assert np.linalg.norm(gx - gx_o) < tol * np.linalg.norm(gx_o)
    assert np.linalg.norm(gv - gv_o) < tol * np.linalg.norm(gv_o)


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
