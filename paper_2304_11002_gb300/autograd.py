"""torch.autograd integration of the solver: phi, g = fmm_forces(rho, solver).

The backward pass calls the library's hand-written adjoint (octo_fmm_backward):
the reverse of L2P, L2L, M2L with the angular-momentum correction, P2P, M2M and
P2M, including the dependence of the centre-of-mass expansion centres on rho.
The adjoint always runs in float64 from the handle's stored forward state, so a
backward must follow the forward it differentiates on the same handle (checked).
"""
from __future__ import annotations

import torch

from . import binding


class OctoFMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho: torch.Tensor, solver: "binding.OctoFMM"):
        if rho.dtype != torch.float64 or rho.numel() != solver.n_leaf_cells or not rho.is_cuda:
            raise ValueError(f"rho must be a float64 CUDA tensor of {solver.n_leaf_cells} elements "
                             f"(got {rho.dtype}, {rho.numel()} elements, on {rho.device})")
        rho = rho.detach().contiguous()
        phi, g = solver.forces(rho)
        solver._forward_id = getattr(solver, "_forward_id", 0) + 1
        ctx.solver = solver
        ctx.forward_id = solver._forward_id
        return phi, g

    @staticmethod
    def backward(ctx, dphi: torch.Tensor, dg: torch.Tensor):
        solver = ctx.solver
        if solver._forward_id != ctx.forward_id:
            raise RuntimeError("the solver ran another forward solve after this one; backward needs its state")
        n = solver.n_leaf_cells
        dev = solver_device(dphi, dg)
        dphi = (dphi if dphi is not None else torch.zeros(n, dtype=torch.float64, device=dev)).contiguous()
        dg = (dg if dg is not None else torch.zeros((3, n), dtype=torch.float64, device=dev)).contiguous()
        drho = torch.empty(n, dtype=torch.float64, device=dphi.device)
        binding.octo_fmm_backward(solver.handle, dphi, dg, drho)
        return drho, None


def solver_device(*ts):
    for t in ts:
        if t is not None:
            return t.device
    return torch.device("cuda")


def fmm_forces(rho: torch.Tensor, solver: "binding.OctoFMM"):
    """Differentiable solve: returns (phi [n_leaf*512], g [3, n_leaf*512])."""
    return OctoFMMFunction.apply(rho, solver)
