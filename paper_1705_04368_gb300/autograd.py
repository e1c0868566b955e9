"""torch.autograd access to the soft-binned MDLG occupations and their adjoint.

``soft_mdlg(x0, v0, eps, sigma, params, nsteps, ckpt_every, width)`` returns the
soft occupations ftilde_i (Q = (2V+1)^2 values, see mdlg_adjoint in
include/mdlg.h) of the interval [0, nsteps] of the Lennard-Jones trajectory
started from (x0, v0); backward() calls mdlg_adjoint with the incoming gradient
as the loss weights, so any loss built from ftilde (moments such as
sum_i |v_i|^2 ftilde_i) is differentiated with respect to x0, v0, eps and sigma
by the hand-written GPU adjoint (segments recomputed from checkpoints).
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np
import torch

from .binding import Params, Simulation


class _SoftMDLG(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, eps, sigma, params, nsteps, ckpt_every, width):
        p = replace(params, eps=float(eps), sigma=float(sigma), sort_every=int(ckpt_every))
        xs = x0.detach().cpu().double().numpy()
        vs = v0.detach().cpu().double().numpy()
        with Simulation(p, xs, vs) as sim:
            out = sim.adjoint(nsteps, ckpt_every, width)
        ctx.save_for_backward(x0, v0, eps, sigma)
        ctx.cfg = (p, nsteps, ckpt_every, width)
        return torch.from_numpy(out["ftilde"]).to(x0.dtype)

    @staticmethod
    def backward(ctx, grad_ft):
        x0, v0, eps, sigma = ctx.saved_tensors
        p, nsteps, ckpt_every, width = ctx.cfg
        with Simulation(p, x0.detach().cpu().double().numpy(),
                        v0.detach().cpu().double().numpy()) as sim:
            out = sim.adjoint(nsteps, ckpt_every, width,
                              dloss=grad_ft.detach().cpu().double().numpy())
        gx = torch.from_numpy(out["grad_x0"]).to(x0.dtype)
        gv = torch.from_numpy(out["grad_v0"]).to(v0.dtype)
        ge = torch.tensor(out["grad_eps"], dtype=eps.dtype)
        gs = torch.tensor(out["grad_sigma"], dtype=sigma.dtype)
        return gx, gv, ge, gs, None, None, None, None


def soft_mdlg(x0, v0, eps, sigma, params: Params, nsteps: int, ckpt_every: int, width: float):
    """Soft f_i of the interval [0, nsteps]; differentiable in x0, v0, eps, sigma."""
    return _SoftMDLG.apply(x0, v0, eps, sigma, params, int(nsteps), int(ckpt_every), float(width))
