"""torch.autograd.Function around the trace estimator and its hand-written adjoint.

TraceFn.apply(kappa, U, context, method, dilution, N, d, seed, prec, tol) returns
the real parts of the estimate of O(t) = tr[g5 D^{-1}(t,t)] per timeslice
(Eq. 21) as a differentiable function of kappa (0-dim float64 tensor) and the
links U (complex128 CUDA tensor [4][T][Z][Y][X][3][3]).  Forward: wd_update_gauge
+ trace_estimate.  Backward: trace_gradient with the incoming per-timeslice
gradients as weights -- one adjoint solve per RHS through gamma5-hermiticity
(none for equal weights) and the link-force kernel.  Both run in libwd; this
module only marshals arguments.
"""
import ctypes

import torch

from ._lib import lib, check, WD_TR_G5_DINV
from .api import trace_estimate, trace_gradient


class TraceFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, U, context, method, dilution, N, d, seed, prec, tol):
        if not (U.is_cuda and U.dtype == torch.complex128 and U.is_contiguous()):
            raise TypeError('U must be a contiguous complex128 CUDA tensor')
        k = float(kappa)
        check(lib.wd_update_gauge(context.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_double(k)), 'wd_update_gauge')
        r = trace_estimate(context.h, method, dilution, N, context.T, d=d, seed=seed, op=WD_TR_G5_DINV, prec=prec,
                           tol=tol)
        ctx.context, ctx.args = context, (method, dilution, N, d, seed, prec, tol)
        ctx.kappa, ctx.U = k, U
        return torch.tensor(r['estimate'].real, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, grad_out):
        method, dilution, N, d, seed, prec, tol = ctx.args
        c = ctx.context
        check(lib.wd_update_gauge(c.h, ctypes.c_void_p(ctx.U.data_ptr()), ctypes.c_double(ctx.kappa)), 'wd_update_gauge')
        w = grad_out.detach().double().cpu().numpy()
        dk, G, H = trace_gradient(c.h, method, dilution, N, c.T, d=d, seed=seed, op=WD_TR_G5_DINV, prec=prec, tol=tol,
                                  weights=w, link_shape=tuple(ctx.U.shape))
        gU = (G + H).conj().transpose(-1, -2).contiguous()
        return (torch.tensor(dk, dtype=torch.float64), gU) + (None,) * 8
