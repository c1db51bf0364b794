"""Differentiable Symanzik action: a torch.autograd.Function whose forward
is the action kernel and whose backward is the force kernel.

S is taken as a function of the algebra parameters omega of a left
perturbation of fixed base links, U = exp(i omega.T) U0 (Eq. 18_1_29_3).  The
backward evaluates the force at U (the left derivative of Eqs. 18_7_25_1 /
18_7_26_1, computed by the staple kernels) and maps it to dS/domega with the
chain rule through the exponential (lqcd_omega_gradient); at omega = 0 the
gradient is minus the force.  Everything runs in liblqcd's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import lqcd


class SymanzikAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, omega: torch.Tensor, base_links: torch.Tensor, lat: lqcd.Lattice):
        om = omega.detach().contiguous()
        U = base_links.detach().clone()
        lqcd.md_update_links(lat, U, om, 1.0)  # U = exp(i omega.T) U0
        S = lqcd.gauge_action(lat, U)
        ctx.lat = lat
        ctx.save_for_backward(om, U)
        return S

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        om, U = ctx.saved_tensors
        lat = ctx.lat
        f = lqcd.gauge_force(lat, U)
        g = lqcd.omega_gradient(lat, om, f)
        return g * grad_out.to(g.dtype), None, None


def symanzik_action(omega: torch.Tensor, base_links: torch.Tensor,
                    lat: lqcd.Lattice) -> torch.Tensor:
    """S_G(exp(i omega.T) U0) as a differentiable FP64 scalar."""
    return SymanzikAction.apply(omega, base_links, lat)
