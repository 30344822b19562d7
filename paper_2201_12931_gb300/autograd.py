"""Differentiable compliance rho -> C through the hand-written adjoint.

Forward: rho~ = H x (density filter kernel), set_density, solve K(rho~) u = f,
C = sum_e E(rho~_e) u_e^T K0 u_e.  Backward: the compliance is self-adjoint
(K u* = dc/du = f gives u* = u, Eq. sensitivity), so the element kernel gives
dC/drho~_e = -p rho~_e^(p-1) (E0 - Emin) u_e^T K0 u_e from the stored state,
and the filter-transpose kernel maps it to dC/dx = H^T dC/drho~.

The grid holds the state of the last forward solve; backward must run before
the next operation that changes the grid's state (checked).
"""
from __future__ import annotations

import torch

from .api import TopoError, TopoGrid
from . import _lib as L


class TopoCompliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, grid: TopoGrid, rmin: float, rel_tol: float = 1e-10, max_it: int = 2000):
        rho = grid.filter(rmin, x.contiguous())
        grid.set_density(rho)
        _, res = grid.solve(rel_tol, max_it)
        if res.status != L.TOPO_OK:
            raise TopoError(res.status, f"state solve did not converge (relres {res.relres:.3e})")
        C, _ = grid.compliance_and_sensitivity()
        ctx.grid = grid
        ctx.rmin = rmin
        ctx.generation = grid.generation
        return x.new_tensor(C)

    @staticmethod
    def backward(ctx, gC):
        grid: TopoGrid = ctx.grid
        if grid.generation != ctx.generation:
            raise RuntimeError("grid state changed between forward and backward of TopoCompliance")
        dc = torch.empty(grid.ne, dtype=torch.float64, device=gC.device)
        grid.compliance_and_sensitivity(dc)
        dx = grid.filter(ctx.rmin, dc, transpose=True)
        return gC * dx, None, None, None, None


def compliance(x: torch.Tensor, grid: TopoGrid, rmin: float, rel_tol: float = 1e-10, max_it: int = 2000):
    return TopoCompliance.apply(x, grid, rmin, rel_tol, max_it)
