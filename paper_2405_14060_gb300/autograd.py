"""log Z as a differentiable function of the log factor tables.

``log_partition(model, log_tables, evid)`` returns log p(e_b) for every
evidence set b.  Its gradient with respect to ``log_tables`` is the factor
marginal p(scope_f = x | e_b) (Thm. "Tensor network differentiation": the
derivative of the contraction with respect to one tensor is the contraction
of the rest), computed by libtn's adjoint pass in the same call as the
forward pass.  The exponentiation of the log tables happens in libtn's leaf
kernel; this module only marshals tensors and applies the chain rule over
the evidence sets.
"""
from __future__ import annotations

import torch

from . import tn as _tn


class LogPartition(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_tables: torch.Tensor, model: "_tn.Model", evid: torch.Tensor,
                prec: str = "fp64"):
        if not log_tables.is_cuda or log_tables.dtype != torch.float64:
            raise TypeError("log_tables must be a float64 CUDA tensor")
        evid = evid.to(device=log_tables.device, dtype=torch.int32).contiguous()
        if evid.dim() == 1:
            evid = evid[None, :]
        nb = evid.shape[0]
        ncard = int(model.card.sum())
        ntab = int(model.table_sizes.sum())
        dev = log_tables.device
        logz = torch.empty(nb, dtype=torch.float64, device=dev)
        marg = torch.empty(nb, ncard, dtype=torch.float64, device=dev)
        grad = torch.empty(nb, ntab, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev).cuda_stream
        model.mar_dev(evid, logz, marg, grad=grad, tables=log_tables.detach().contiguous(),
                      tables_are_log=True, prec=prec, stream=stream)
        ctx.save_for_backward(grad)
        ctx.mark_non_differentiable(marg)
        return logz, marg

    @staticmethod
    def backward(ctx, g_logz, g_marg):
        (grad,) = ctx.saved_tensors
        return (g_logz[:, None] * grad).sum(0), None, None, None


def log_partition(model, log_tables, evid, prec="fp64"):
    """(log Z per evidence set, marginals per evidence set); differentiable in
    ``log_tables`` through log Z."""
    return LogPartition.apply(log_tables, model, evid, prec)
