"""Compliance of a design as a differentiable PyTorch function.

c(rho) = q^T t with K(F rho) t = q (Eq. 3-5).  The forward pass filters the
design (Eq. 6-8), forms the SIMP conductivities (Eq. 4) and solves with MGCG;
the backward pass is the adjoint sensitivity (Eq. 9-11).  The problem is
self-adjoint, so the adjoint solution is -t and
dc/drho = F^T(-p (k0 - kmin) rho~^(p-1) t_e^T k0 t_e) needs no second solve:
the library returns it with the compliance.  Every step runs in the
library's kernels; PyTorch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import mgar


class ComplianceFunction(torch.autograd.Function):
    """c = compliance(rho); T is the temperature buffer (warm start in,
    solution out)."""

    @staticmethod
    def forward(ctx, rho, solver, T):
        rho_c = rho.detach().contiguous()
        solver.set_density(rho_c, physical=False)
        solver.solve_mgcg(T)
        dc = torch.empty_like(rho_c)
        c = solver.sensitivity(T, dc)
        ctx.save_for_backward(dc)
        return torch.tensor(c, dtype=rho.dtype, device=rho.device)

    @staticmethod
    def backward(ctx, grad):
        (dc,) = ctx.saved_tensors
        return grad * dc, None, None


class Compliance(torch.nn.Module):
    """Holds a solver handle and its warm-start temperatures:
    Compliance(params, fixed, q)(rho) is the compliance of design rho, and
    backward() gives its gradient with respect to rho."""

    def __init__(self, params: mgar.Params, fixed, q, stream=None):
        super().__init__()
        self.solver = mgar.Solver(params, fixed, q, stream=stream)
        self.T = None

    def forward(self, rho):
        if self.T is None:
            self.T = torch.zeros(self.solver.n_nodes, dtype=torch.float64, device=rho.device)
        return ComplianceFunction.apply(rho, self.solver, self.T)

    def close(self):
        self.solver.close()
