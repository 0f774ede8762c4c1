"""Differentiable grid integration: V_mu,nu(R) as a torch.autograd.Function.

forward(V, tau) -> H runs gint_vlocal.  backward(gH) runs gint_vlocal_backward, i.e. the
adjoint density kernel for dL/dV(r) = dV * rho[sym(gH)](r) and the grad-phi (Pulay) kernel for
dL/dtau_I (Eq. force_lcao with V(r) held fixed, Sec. IV.D), both hand-written CUDA; torch only
holds the buffers.  sym(G) is the block-symmetric part (G_mu,nu(R) + G_nu,mu(-R)) / 2; only
that part of gH reaches V_mu,nu because V_mu,nu(R) = V_nu,mu(-R).
"""
from __future__ import annotations

import numpy as np
import torch

from . import gint as G


def _move_to(handle, tau_h):
    """Put the handle's atoms at tau_h (flat float64) if they are elsewhere."""
    if getattr(handle, "_tau", None) is None or not np.array_equal(handle._tau, tau_h):
        G.gint_update_positions(handle, tau_h)
        handle._tau = tau_h.copy()


class GintVlocal(torch.autograd.Function):
    """H = vlocal(V; tau).  `tau` (natoms x 3, float64) selects the atom positions: if they
    differ from the handle's, the handle is moved with gint_update_positions (same neighbour
    topology required).  The positions of each forward are kept with its graph node, and the
    backward moves the handle back to them if another forward moved it in between, so every
    gradient is taken at the geometry of its own forward."""

    @staticmethod
    def forward(ctx, V, tau, handle, prec="fp64"):
        tau_h = tau.detach().to("cpu", torch.float64).numpy().reshape(-1).copy()
        _move_to(handle, tau_h)
        Vc = V.detach().contiguous()
        H = torch.empty(handle.nvalues, dtype=torch.float64, device=V.device)
        G.gint_vlocal(handle, Vc, H, prec)
        ctx.save_for_backward(Vc)
        ctx.handle, ctx.prec, ctx.tau_device, ctx.tau_h = handle, prec, tau.device, tau_h
        return H

    @staticmethod
    def backward(ctx, gH):
        (V,) = ctx.saved_tensors
        h = ctx.handle
        need_v, need_tau = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gV = torch.empty_like(V) if need_v else None
        gt = torch.empty(3 * h.natoms, dtype=torch.float64, device=V.device) if need_tau else None
        if need_v or need_tau:
            _move_to(h, ctx.tau_h)
            G.gint_vlocal_backward(h, V, gH.contiguous(), gV, gt, ctx.prec)
        if gt is not None:
            gt = gt.view(-1, 3).to(ctx.tau_device)
        return gV, gt, None, None


def vlocal(V, tau, handle, prec="fp64"):
    return GintVlocal.apply(V, tau, handle, prec)
