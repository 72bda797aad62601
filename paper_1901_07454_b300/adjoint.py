"""Voltage-loss fitting through the library's discrete adjoint (arb_adjoint).

AdjointLoss is a torch.autograd.Function of the per-group densities
theta [n_groups, 4] = (gnabar, gkbar, gl in S/cm^2, cm in uF/cm^2): its forward runs the
implicit step on the GPU from the model's initial state and returns the loss
  L = loss_scale * sum_s sum_o (V_{obs_cv[o]}(t_{s+1}) - target[s, o])^2,
its backward returns dL/dtheta computed by the reverse sweep (checkpointed every
checkpoint_every steps). Only argument marshalling happens here: theta is spread over the
model's per-CV and per-instance arrays, every step runs in the CUDA library.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from .sim import Simulation


def spread_params(model, group_of_cv, theta):
    """Copy of `model` whose gnabar, gkbar, gl (per HH instance) and cm (per CV) are the values
    of their CV's group in theta [n_groups, 4]; CVs of group -1 keep their own values."""
    theta = np.asarray(theta, np.float64)
    group = np.asarray(group_of_cv, np.int64)
    m = copy.copy(model)
    hg = group[np.asarray(model.hh_cv, np.int64)]
    for name, col in (("gnabar", 0), ("gkbar", 1), ("gl", 2)):
        v = np.array(getattr(model, name), np.float64, copy=True)
        v[hg >= 0] = theta[hg[hg >= 0], col]
        setattr(m, name, v)
    cm = np.array(model.cm, np.float64, copy=True)
    cm[group >= 0] = theta[group[group >= 0], 3]
    m.cm = cm
    return m


class AdjointLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, model, group_of_cv, obs_cv, target, loss_scale, n_steps, dt=0.025,
                checkpoint_every=500, device="cuda"):
        th = theta.detach().to("cpu", torch.float64).numpy()
        m = spread_params(model, group_of_cv, th)
        sim = Simulation(m, dt=dt, device=device)
        loss, grad = sim.adjoint(n_steps, obs_cv, target, loss_scale, group_of_cv, th.shape[0], checkpoint_every)
        ctx.save_for_backward(grad.to(theta.device, theta.dtype))
        return torch.tensor(loss, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g * grad,) + (None,) * 9


def adjoint_loss(theta, model, group_of_cv, obs_cv, target, loss_scale, n_steps, dt=0.025, checkpoint_every=500,
                 device="cuda"):
    return AdjointLoss.apply(theta, model, group_of_cv, obs_cv, target, loss_scale, n_steps, dt, checkpoint_every,
                             device)
