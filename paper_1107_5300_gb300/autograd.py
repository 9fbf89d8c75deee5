"""``torch.autograd.Function`` over the conductance entry points.

Forward: T(E_c) for every energy of one ribbon whose on-site energies are the
input tensor (rgf_conductance).  Backward: rgf_conductance_grad (the
two-sided gradient sweep) gives dT_c/d eps for every site; the vector-Jacobian
product sums them with the incoming weights.  All numerics run in librgf.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rgf


class RGFConductance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, E, N, t=-2.7, removed=None, eta_device=1e-8, eta_lead=1e-8,
                precision=rgf.RGF_FP64, ckpt_stride=0):
        L = eps.shape[0]
        e_host = eps.detach().to("cpu", torch.float64).numpy()
        E_host = np.ascontiguousarray(E.detach().to("cpu", torch.float64).numpy())
        rem = None if removed is None else np.ascontiguousarray(removed, dtype=np.uint8)
        rib = rgf.Ribbon(N, L, t, onsite=e_host, removed=rem)
        T, _ = rgf.conductance([rib] * E_host.size, E_host, eta_device, eta_lead, precision)
        ctx.args = (N, L, t, e_host, rem, E_host, eta_device, eta_lead, precision, ckpt_stride)
        ctx.device = eps.device
        return torch.as_tensor(T, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, gT):
        N, L, t, e_host, rem, E_host, etad, etal, prec, stride = ctx.args
        rib = rgf.Ribbon(N, L, t, onsite=e_host, removed=rem)
        _, g, _ = rgf.conductance_grad([rib] * E_host.size, E_host, etad, etal, prec, stride)
        w = gT.detach().to("cpu", torch.float64).numpy()
        grad = np.tensordot(w, g, axes=(0, 0))
        return (torch.as_tensor(grad, dtype=torch.float64, device=ctx.device),
                None, None, None, None, None, None, None, None)


def conductance(eps, E, N, **kw):
    """T(E) of the ribbon with on-site energies ``eps`` [L, 2N], differentiable in eps."""
    return RGFConductance.apply(eps, E, N, kw.get("t", -2.7), kw.get("removed"),
                                kw.get("eta_device", 1e-8), kw.get("eta_lead", 1e-8),
                                kw.get("precision", rgf.RGF_FP64), kw.get("ckpt_stride", 0))
