"""The dual bound as a differentiable PyTorch function of the pair costs.

    lbs = dual_bounds([d1, d2, ...], [(TX1, TY1), ...], [allowed1, ...], iters=50)
    loss = -lbs.sum(); loss.backward()        # d1.grad, d2.grad from the adjoint kernels

Forward builds one device store for all pairs (host compiler, candidate masks held fixed),
runs the iterations with a checkpoint every `checkpoint_every` of them (disco_record) and
returns each pair's bound. Backward runs the adjoint of the recorded iterations on the
device (disco_grad) and scales each pair's gradient by the incoming one. Argument
marshalling only: every step runs in the CUDA library.
"""
from __future__ import annotations

import torch

from .api import Solver


class _DualBounds(torch.autograd.Function):
    @staticmethod
    def forward(ctx, meta, *costs):
        meshes, allowed, iters, every, opts = meta
        pairs = [(TX, TY, d.detach().contiguous().float(), a) for d, (TX, TY), a in zip(costs, meshes, allowed)]
        s = Solver.batch(pairs, **opts)
        s.record(iters, every)
        lbs = s.lower_bounds()
        ctx.solver = s
        ctx.shapes = [tuple(d.shape) for d in costs]
        ctx.device = costs[0].device
        return torch.from_numpy(lbs).to(costs[0].device)

    @staticmethod
    def backward(ctx, g):
        s = ctx.solver
        n = sum(a * b for a, b in ctx.shapes)
        flat = torch.empty(n, dtype=torch.float32, device=ctx.device)
        torch.cuda.current_stream(ctx.device).synchronize()
        s.grad(flat)
        s.close()
        ctx.solver = None
        out, o = [], 0
        g = g.to(torch.float32)
        for i, (a, b) in enumerate(ctx.shapes):
            out.append(flat[o:o + a * b].view(a, b) * g[i])
            o += a * b
        return (None, *out)


def dual_bounds(costs, meshes, allowed, iters: int, checkpoint_every: int = 10, **opts) -> torch.Tensor:
    """Per-pair dual bounds after `iters` iterations (float64 tensor), differentiable in the
    pair-cost tensors `costs` (CUDA float32, one (nvx, nvy) per pair). `meshes` = [(TX, TY)]
    triangle arrays, `allowed` = candidate masks (uint8, or None for the full space)."""
    meta = (list(meshes), [None if a is None else a for a in allowed], int(iters), int(checkpoint_every), opts)
    return _DualBounds.apply(meta, *costs)
