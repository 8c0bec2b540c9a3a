"""torch.autograd wrapper of the mW forces and their adjoint (force matching).

``ForceField(n, box)`` owns one libmw system (a single box, or a batch of
boxes such as the frames of a force-matching set).  ``ForceField.forces(x,
theta)`` returns the FP32 forces of positions ``x`` (n_total x 3, float64,
CUDA) for parameters ``theta = (lambda, epsilon, sigma)``; its backward pass
calls the CUDA adjoint (mw_energy_forces_vjp), which recomputes the leg and
triplet terms instead of storing them, and returns dL/dx and dL/dtheta.
Torch provides device memory and streams only; the arithmetic runs in libmw.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch

from . import mw


class _MWForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, theta: torch.Tensor, ff: "ForceField"):
        ff._set_theta(theta)
        x = x.detach().to(torch.float64).contiguous()
        f = torch.empty(x.shape, dtype=torch.float32, device=x.device)
        ff.stream.wait_stream(torch.cuda.current_stream(x.device))
        mw.mw_energy_forces_dev(ff.system.h, x, f, ff.energy, ff.virial)  # synchronises the system stream
        ctx.ff = ff
        ctx.theta_dtype = theta.dtype
        ctx.theta_device = theta.device
        return f

    @staticmethod
    def backward(ctx, gf: torch.Tensor):
        ff = ctx.ff
        gf = gf.detach().to(torch.float32).contiguous()
        gx = torch.empty_like(gf)
        ff.stream.wait_stream(torch.cuda.current_stream(gf.device))
        gth = mw.mw_energy_forces_vjp(ff.system.h, gf, gx, ff.nbox)  # per box (lambda, epsilon, sigma)
        gtheta = torch.as_tensor(gth.sum(0), dtype=ctx.theta_dtype, device=ctx.theta_device)
        return gx.to(torch.float64), gtheta, None


class ForceField:
    """mW forces with autograd for one box (n: int) or a batch (n: list of ints)."""

    def __init__(self, n, box, skin: float = 1.0, mass: float = 18.015, device: Optional[torch.device] = None):
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.Stream(self.device)
        self.system = mw.System(n, box, mass=mass, skin=skin, stream=self.stream.cuda_stream)
        self.nbox = self.system.nbox
        self.energy = torch.zeros((self.nbox, 3), dtype=torch.float64, device=self.device)
        self.virial = torch.zeros((self.nbox, 6), dtype=torch.float64, device=self.device)
        self._theta = None

    def _set_theta(self, theta: torch.Tensor):
        t = tuple(float(v) for v in theta.detach().cpu().tolist())
        if t != self._theta:
            p = mw.mw_params_default()
            p.lambda_, p.epsilon, p.sigma = t
            self.system.set_params(p)
            self._theta = t

    def forces(self, x: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
        return _MWForces.apply(x, theta, self)

    def close(self):
        self.system.close()


def force_matching_loss(f: torch.Tensor, f_target: torch.Tensor) -> torch.Tensor:
    """L = mean over atoms and components of (F - F*)^2 (sum over frames / (3 N F))."""
    return ((f.to(torch.float64) - f_target.to(torch.float64)) ** 2).mean()


def paper_theta(device=None, dtype=torch.float64) -> torch.Tensor:
    """(lambda, epsilon, sigma) of the mW model (Sec. II.D)."""
    p = mw.mw_params_default()
    return torch.tensor([p.lambda_, p.epsilon, p.sigma], dtype=dtype, device=device)
