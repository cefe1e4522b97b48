"""torch.autograd.Function around gpf_radiance_fwd / gpf_radiance_bwd. The
forward rebuilds the index for the current parameters and hit points, the
backward recomputes the exponentials instead of storing per-pair weights."""

from __future__ import annotations

import math

import torch

from .api import (GPF_SUM, PAPER_EPS, Field, Index, Queries, gpf_radiance_bwd,
                  gpf_radiance_fwd)


class GPFRadiance(torch.autograd.Function):
    """out = GPFRadiance.apply(mean, quat, logscale, spectrum, index, queries,
    mode, r_max, eps): radiance [C,M] at the hit points; gradients flow to the
    four parameter tensors."""

    @staticmethod
    def forward(ctx, mean, quat, logscale, spectrum, index: Index, queries: Queries,
                mode: int = GPF_SUM, r_max: float = math.inf, eps: float = PAPER_EPS):
        field = Field(mean, quat, logscale, spectrum)
        index.build(field, queries)
        out, z = gpf_radiance_fwd(index, field, queries, mode, r_max, eps)
        ctx.save_for_backward(mean, quat, logscale, spectrum, out, z)
        ctx.index, ctx.queries, ctx.params = index, queries, (mode, r_max, eps)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        mean, quat, logscale, spectrum, out, z = ctx.saved_tensors
        mode, r_max, eps = ctx.params
        field = Field(mean, quat, logscale, spectrum)
        g = gpf_radiance_bwd(ctx.index, field, ctx.queries, grad_out.contiguous(), out, z, mode,
                             r_max, eps)
        return g.mean, g.quat, g.logscale, g.spectrum, None, None, None, None, None


def gpf_radiance(field: Field, index: Index, queries: Queries, mode: int = GPF_SUM,
                 r_max: float = math.inf, eps: float = PAPER_EPS) -> torch.Tensor:
    return GPFRadiance.apply(field.mean, field.quat, field.logscale, field.spectrum, index,
                             queries, mode, r_max, eps)
