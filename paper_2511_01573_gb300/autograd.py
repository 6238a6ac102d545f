"""Differentiable adaptive integral: a torch.autograd.Function over the C ABI.

forward: the adaptive integration of a built-in family with parameters
(a, u), keeping its final partition (GMQ_KEEP_PARTITION).
backward: the adjoint kernel over that frozen partition (gmq_rule_grad),
which returns the exact gradient of the quadrature sum with respect to a
and u; the partition is not re-adapted, so the result is a smooth function
of the parameters near the point of evaluation.

Works on a single parameter set (a, u of shape [d]) or a batch ([B, d]):
each row is its own integral with its own partition.  Tensors may live on
the CPU or on a CUDA device; the integration always runs on the context's
GPU.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gmq


class FrozenPartitionIntegral(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, u, family, rel_tol, context, max_regions):
        batched = a.dim() == 2
        A = a.detach().to("cpu", torch.float64).reshape(-1, a.shape[-1]).numpy()
        U = u.detach().to("cpu", torch.float64).reshape(-1, u.shape[-1]).numpy()
        vals, parts = [], []
        for ai, ui in zip(A, U):
            r = context.integrate(family, ai, ui, rel_tol, max_regions=max_regions,
                                  keep_partition=True)
            if r.status not in (gmq.OK, gmq.MAX_ITERS, gmq.CAP_REACHED, gmq.ROUNDOFF_LIMIT):
                raise gmq.GmqError("gmq_integrate", r.status)
            vals.append(r.integral)
            parts.append(context.partition_copy())
        ctx.family = family
        ctx.context = context
        ctx.params = (A, U)
        ctx.parts = parts
        ctx.batched = batched
        out = torch.tensor(vals, dtype=torch.float64, device=a.device)
        return out if batched else out[0]

    @staticmethod
    def backward(ctx, grad_out):
        A, U = ctx.params
        ga = np.zeros_like(A)
        gu = np.zeros_like(U)
        for i, (ai, ui) in enumerate(zip(A, U)):
            c, h = ctx.parts[i]
            g, _ = ctx.context.rule_grad(ctx.family, ai, ui, c, h)
            d = len(ai)
            ga[i] = g[:d]
            gu[i] = g[d:]
        go = grad_out.detach().to("cpu", torch.float64).reshape(-1, 1).numpy()
        ga = torch.tensor(go * ga, dtype=torch.float64, device=grad_out.device)
        gu = torch.tensor(go * gu, dtype=torch.float64, device=grad_out.device)
        if not ctx.batched:
            ga, gu = ga[0], gu[0]
        return ga, gu, None, None, None, None


def integral(a, u, family=gmq.GAUSSIAN, rel_tol=1e-8, context=None, max_regions=1 << 22):
    """I(a, u) of a built-in family over [0,1]^d, differentiable in a and u
    through the frozen final partition."""
    if context is None:
        raise ValueError("pass a gmq.Context")
    return FrozenPartitionIntegral.apply(a, u, family, rel_tol, context, max_regions)
