"""torch.autograd.Function over the overlap cost and its hand-written adjoint.

``OverlapAlign.apply(items, params)`` returns f[P] for every pair i < j of a
2-D cloud set, the second item of each pair moved by its (theta, tx, ty);
backward calls the library's adjoint kernel, which recomputes the
exponentials instead of storing them.  ``OverlapAlignList.apply(items, pi,
pj, params)`` does the same for a chosen list of pairs (pj[k] moved).
"""
from __future__ import annotations

import torch

from .binding import AP_FN_OVERLAP, Items


class OverlapAlign(torch.autograd.Function):
    @staticmethod
    def forward(ctx, items: Items, params: torch.Tensor):
        params = params.detach().contiguous().float()
        ctx.items = items
        ctx.save_for_backward(params)
        return items.run_pairs(AP_FN_OVERLAP, params=params)

    @staticmethod
    def backward(ctx, grad_f):
        (params,) = ctx.saved_tensors
        g, _ = ctx.items.backward(params=params, grad_out=grad_f.contiguous().float())
        return None, g


def overlap_align(items: Items, params: torch.Tensor) -> torch.Tensor:
    return OverlapAlign.apply(items, params)


class OverlapAlignList(torch.autograd.Function):
    @staticmethod
    def forward(ctx, items: Items, pi, pj, params: torch.Tensor):
        params = params.detach().contiguous().float()
        ctx.items, ctx.pi, ctx.pj = items, pi, pj
        ctx.save_for_backward(params)
        return items.run_pairs_list(pi, pj, AP_FN_OVERLAP, params=params)

    @staticmethod
    def backward(ctx, grad_f):
        (params,) = ctx.saved_tensors
        g, _ = ctx.items.backward_list(ctx.pi, ctx.pj, params=params,
                                       grad_out=grad_f.contiguous().float())
        return None, None, None, g


def overlap_align_list(items: Items, pi, pj, params: torch.Tensor) -> torch.Tensor:
    return OverlapAlignList.apply(items, pi, pj, params)
