"""Gradients of a loss on the final order parameter through the library's
discrete adjoint (C ABI ``lbm_adjoint_*``), as a ``torch.autograd.Function``.

``rollout(phi0, sigma, M, shape=..., nsteps=..., **params)`` advances the
initial field ``phi0`` (CUDA float64 tensor, shape ``(ny, nx)``) by
``nsteps`` D2Q9 steps with surface tension ``sigma`` and mobility ``M``
(0-d tensors) and returns the final phi.  Its backward pass replays the run
from checkpoints every ``checkpoint_every`` steps and returns dL/dphi0,
dL/dsigma and dL/dM.  All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import capi
from .sim import Simulation


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, sigma, M, shape, nsteps, checkpoint_every, precision, params):
        prm = dict(params)
        prm.update(sigma=float(sigma), M=float(M))
        stream = torch.cuda.current_stream().cuda_stream
        sim = Simulation(shape, precision=precision, stream=stream, **prm)
        rc, h = capi.lbm_adjoint_create(sim.handle, checkpoint_every, max(nsteps, 1))
        capi.check(rc, "lbm_adjoint_create")
        phi0 = phi0.detach().contiguous()
        capi.check(capi.lbm_adjoint_forward(h, phi0, 1, nsteps), "lbm_adjoint_forward")
        out = torch.empty_like(phi0)
        sim.moments_device(phi=out)
        ctx.sim, ctx.adj = sim, h
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.detach().to(torch.float64).contiguous()
        d_phi0 = torch.empty_like(g)
        rc, grads = capi.lbm_adjoint_backward(ctx.adj, g, 1, d_phi0)
        capi.check(rc, "lbm_adjoint_backward")
        capi.lbm_adjoint_destroy(ctx.adj)
        ctx.sim.close()
        dev = g.device
        return (d_phi0, torch.tensor(grads[0], dtype=torch.float64, device=dev),
                torch.tensor(grads[1], dtype=torch.float64, device=dev),
                None, None, None, None, None)


def rollout(phi0, sigma, M, *, shape, nsteps, checkpoint_every=100, precision="fp64",
            **params):
    """Differentiable run of the phase-field LBM (see module docstring)."""
    return _Rollout.apply(phi0, sigma, M, tuple(shape), int(nsteps), int(checkpoint_every),
                          precision, params)
