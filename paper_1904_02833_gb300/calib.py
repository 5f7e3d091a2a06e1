"""Differentiable rollouts for calibration: the library's adjoint wrapped in
torch.autograd.Function.

theta [n_snakes, 5] = (bend compliance, damping, tau_inflate, tau_deflate, curvature gain)
per snake; the rollout returns the last node's position after every env-step
[n_steps, n_snakes, 3].  Backward runs the library's adjoint kernels (checkpoint every
`ckpt_every` env-steps, recompute, reverse sweep); nothing is differentiated by torch
except the loss the caller builds on the tips.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


class SnakeRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, sim, n_steps, ckpt_every):
        theta = theta.detach().to(device=sim.device, dtype=torch.float32).contiguous()
        tips = torch.empty(n_steps, sim.n, 3, device=sim.device, dtype=torch.float32)
        N.check(sim.lib.sim_calib_forward(sim.h, _p(theta), int(n_steps), int(ckpt_every), _p(tips)))
        ctx.sim = sim
        return tips

    @staticmethod
    def backward(ctx, tips_bar):
        sim = ctx.sim
        tb = tips_bar.to(dtype=torch.float32).contiguous()
        grad = torch.empty(sim.n, 5, device=sim.device, dtype=torch.float32)
        N.check(sim.lib.sim_calib_backward(sim.h, _p(tb), _p(grad)))
        return grad, None, None, None


def rollout(sim, theta: torch.Tensor, n_steps: int, ckpt_every: int = 20) -> torch.Tensor:
    """Tips [n_steps, n_snakes, 3] of a differentiable rollout from sim's current state."""
    return SnakeRollout.apply(theta, sim, n_steps, ckpt_every)


def theta_of(w: dict) -> torch.Tensor:
    """theta [n, 5] from a workload dict (alpha_b, damping, tau_inf, tau_def, gain)."""
    import numpy as np
    return torch.tensor(np.stack([w["alpha_b"], w["damping"], w["tau_inf"], w["tau_def"], w["gain"]], 1),
                        dtype=torch.float32)
