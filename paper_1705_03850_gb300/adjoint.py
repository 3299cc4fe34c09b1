"""Differentiable DEM rollouts: torch.autograd.Function over the C ABI.

Forward: set the per-instance material {E, e, mu}, load the initial state, run
the rollout with checkpoints (lists frozen) and return the observables
{kinetic energy, runout} per instance.  Backward: the hand-written adjoint of
the contact law and the integrator in the CUDA library, seeded with the
incoming gradient of the observables.
"""
from __future__ import annotations

import numpy as np
import torch

from . import dem


class DEMRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, sim, state, nsteps, checkpoint_every, axis):
        p = params.detach().to("cpu", torch.float64).numpy()
        sim.set_material(p)
        sim.write_state(*state)
        sim.rollout_forward(nsteps, checkpoint_every)
        obs = sim.observables(axis)
        ctx.sim = sim
        ctx.axis = np.asarray(axis, dtype=np.float64)
        return torch.as_tensor(obs, dtype=params.dtype, device=params.device)

    @staticmethod
    def backward(ctx, grad_obs):
        w = grad_obs.detach().to("cpu", torch.float64).numpy()
        g = ctx.sim.rollout_adjoint(w, ctx.axis)
        return torch.as_tensor(g, dtype=grad_obs.dtype, device=grad_obs.device), None, None, None, None, None


def rollout(params, sim, state, nsteps, checkpoint_every, axis):
    """Observables (B, 2) of a rollout, differentiable with respect to params (B, 3) = {E, e, mu}."""
    return DEMRollout.apply(params, sim, state, nsteps, checkpoint_every, axis)
