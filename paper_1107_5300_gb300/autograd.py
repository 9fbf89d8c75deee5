"""``torch.autograd.Function`` over the conductance entry points.

Forward: T(E_c) for every energy of one ribbon whose on-site energies are the
input tensor (rgf_conductance_dev, device buffers on the current stream).
Backward: rgf_conductance_grad_dev (the two-sided gradient sweep) with the
incoming cotangent as its chain weights returns the vector-Jacobian product
sum_c gT_c dT_c/d eps directly on the device.  All numerics run in
librgf.so; torch provides the device memory and the stream.
"""
from __future__ import annotations

import torch

from . import rgf


def _ribbon(eps, removed, N, t):
    """A library ribbon copied (device to device) from CUDA tensors."""
    L = eps.shape[0]
    e = eps.detach().to(torch.float64).contiguous()
    r = None if removed is None else torch.as_tensor(removed, dtype=torch.uint8,
                                                     device=eps.device).contiguous()
    stream = torch.cuda.current_stream(eps.device).cuda_stream
    rib = rgf.Ribbon.from_device(N, L, t, e.data_ptr(), r.data_ptr() if r is not None else None,
                                 stream)
    return rib, (e, r)        # keep the sources alive until the stream has copied them


class RGFConductance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, E, N, t=-2.7, removed=None, eta_device=1e-8, eta_lead=1e-8,
                precision=rgf.RGF_FP64, ckpt_stride=0):
        if eps.device.type != "cuda":
            raise ValueError("RGFConductance runs on a CUDA device: pass eps as a CUDA tensor")
        dev = eps.device
        rib, keep = _ribbon(eps, removed, N, t)
        Ed = E.detach().to(device=dev, dtype=torch.float64).contiguous()
        n = Ed.numel()
        T = torch.empty(n, dtype=torch.float64, device=dev)
        st = torch.empty(n, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream(dev).cuda_stream
        rgf.conductance_dev([rib] * n, Ed.data_ptr(), n, T.data_ptr(), st.data_ptr(), eta_device,
                            eta_lead, precision, stream)
        ctx.save_for_backward(Ed)
        ctx.rib, ctx.keep = rib, keep
        ctx.args = (eta_device, eta_lead, precision, ckpt_stride)
        ctx.shape = tuple(eps.shape)
        ctx.status = st
        return T

    @staticmethod
    def backward(ctx, gT):
        (Ed,) = ctx.saved_tensors
        etad, etal, prec, stride = ctx.args
        dev = Ed.device
        n = Ed.numel()
        w = gT.detach().to(device=dev, dtype=torch.float64).contiguous()
        T = torch.empty(n, dtype=torch.float64, device=dev)
        grad = torch.empty(ctx.shape, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev).cuda_stream
        rgf.conductance_grad_dev([ctx.rib] * n, Ed.data_ptr(), n, T.data_ptr(), grad.data_ptr(),
                                 w.data_ptr(), 0, etad, etal, prec, stride, stream)
        return grad, None, None, None, None, None, None, None, None


def conductance(eps, E, N, **kw):
    """T(E) of the ribbon with on-site energies ``eps`` [L, 2N] (a CUDA tensor),
    differentiable in eps."""
    return RGFConductance.apply(eps, E, N, kw.get("t", -2.7), kw.get("removed"),
                                kw.get("eta_device", 1e-8), kw.get("eta_lead", 1e-8),
                                kw.get("precision", rgf.RGF_FP64), kw.get("ckpt_stride", 0))
