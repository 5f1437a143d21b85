"""Spectral-mismatch loss as a torch.autograd.Function whose backward is the
library's hand-written adjoint (graph_reduce_loss_bwd).

Forward keeps only the aggregate means y_0, the fine Rayleigh quotients and
the aggregate sizes; backward recomputes the reduced-graph sweeps from them.
The loss is differentiable with respect to the reduced-graph edge weights w_c
(the quantity the edge-scaling step of Sec. 3.3.3 adjusts).
"""
from __future__ import annotations

import torch

from . import binding as B


class SpectralMismatchLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w_c, fine, coarse, agg, X, sweeps_c, omega):
        loss, saved = B.graph_reduce_loss_fwd(fine, coarse, agg, X, w_c.detach().contiguous(), sweeps_c, omega)
        ctx.save_for_backward(w_c, saved)
        ctx.coarse = coarse
        ctx.K = int(X.shape[1])
        ctx.sweeps_c = int(sweeps_c)
        ctx.omega = float(omega)
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        w_c, saved = ctx.saved_tensors
        g = grad_out.detach().reshape(1).to(torch.float32).contiguous()
        grad_w = B.graph_reduce_loss_bwd(ctx.coarse, saved, ctx.K, w_c.detach().contiguous(), ctx.sweeps_c,
                                         ctx.omega, g)
        return grad_w, None, None, None, None, None, None


def spectral_mismatch_loss(w_c, fine, coarse, agg, X, sweeps_c=5, omega=0.7):
    return SpectralMismatchLoss.apply(w_c, fine, coarse, agg, X, sweeps_c, omega)
