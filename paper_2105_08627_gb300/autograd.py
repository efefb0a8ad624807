"""torch.autograd.Function around the library's port solve and adjoint gradient.

``PortInductance.apply(lam, sigma0, handle, freq, i, j)`` returns the port
inductance L_ij = Im(Zport_ij) / omega (a 0-d float64 tensor) for per-voxel
London depth ``lam`` and normal conductivity ``sigma0`` (float64 tensors of
length K, voxel order); its backward gives dL_ij/dlam and dL_ij/dsigma0 from
the adjoint (svh_grad_inductance), which reuses the forward port solutions.
All computation runs in the library; this is argument marshalling only.
"""
from __future__ import annotations

import numpy as np
import torch


class PortInductance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lam, sigma0, handle, freq, i, j, solve_opts=None):
        lam_np = lam.detach().cpu().numpy().astype(np.float64)
        sig_np = sigma0.detach().cpu().numpy().astype(np.float64)
        handle.set_materials(lam_np, sig_np)
        res = handle.solve([freq], **(solve_opts or {}))
        gl, gs = handle.grad_inductance(i, j)
        ctx.save_for_backward(torch.from_numpy(gl).to(lam.device), torch.from_numpy(gs).to(sigma0.device))
        return torch.tensor(res["L"][0, i, j], dtype=torch.float64, device=lam.device)

    @staticmethod
    def backward(ctx, grad_out):
        gl, gs = ctx.saved_tensors
        return grad_out * gl, grad_out * gs, None, None, None, None, None


def port_inductance(lam, sigma0, handle, freq, i=0, j=0, **solve_opts):
    return PortInductance.apply(lam, sigma0, handle, freq, i, j, solve_opts)
