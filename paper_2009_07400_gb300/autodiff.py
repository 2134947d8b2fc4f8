"""torch.autograd.Function over the library's hand-written adjoint.

``rollout_loss(ctx, eps, sigma, x0, v0, nsteps, window)`` returns the mean
potential energy over the last ``window`` of ``nsteps`` velocity-Verlet steps
started from (x0, v0) with LJ parameters (eps, sigma); its backward pass gives
d loss / d (eps, sigma, x0, v0).  Both passes run in the CUDA library
(``md_adjoint``: checkpointed forward, bit-exact recomputation per block,
reverse sweep with the pair Jacobian-vector product); this module only moves
arrays across the C ABI.  CUDA tensors x0, v0 stay on the device: the state
goes in through ``md_set_state_device`` and the gradients come back through
``md_adjoint_device`` as CUDA tensors; host tensors take the host calls.  The
context keeps its (x0, v0) state afterwards.
"""
from __future__ import annotations

import torch


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, eps, sigma, x0, v0, md_ctx, nsteps, window, ckpt_every):
        md_ctx.set_lj(float(eps), float(sigma))
        if x0.is_cuda and v0.is_cuda:
            md_ctx.set_state_device(x0.detach().double().contiguous(),
                                    v0.detach().double().contiguous())
            loss, ge, gs, gx, gv = md_ctx.adjoint_device(nsteps, window, ckpt_every)
        else:
            md_ctx.set_state(x0.detach().cpu().double().numpy(), v0.detach().cpu().double().numpy())
            loss, ge, gs, gx, gv = md_ctx.adjoint(nsteps, window, ckpt_every)
            gx, gv = torch.from_numpy(gx), torch.from_numpy(gv)
        fctx.grads = (ge, gs, gx, gv)
        fctx.meta = (eps, sigma, x0, v0)
        return torch.tensor(loss, dtype=torch.float64, device=x0.device)

    @staticmethod
    def backward(fctx, gout):
        ge, gs, gx, gv = fctx.grads
        eps, sigma, x0, v0 = fctx.meta
        g = gout.detach().to(torch.float64)
        gx, gv = gx.to(g.device), gv.to(g.device)
        return ((g * ge).to(eps), (g * gs).to(sigma), (g * gx).to(x0), (g * gv).to(v0),
                None, None, None, None)


def rollout_loss(md_ctx, eps, sigma, x0, v0, nsteps, window, ckpt_every=10):
    """Differentiable mean-PE loss of a rollout (see module docstring)."""
    if not torch.is_tensor(eps):
        eps = torch.tensor(float(eps), dtype=torch.float64)
    if not torch.is_tensor(sigma):
        sigma = torch.tensor(float(sigma), dtype=torch.float64)
    return _Rollout.apply(eps, sigma, x0, v0, md_ctx, int(nsteps), int(window), int(ckpt_every))
