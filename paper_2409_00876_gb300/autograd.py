"""Sampled path stress as a differentiable PyTorch function.

``sampled_stress(xy, graph, n_pairs, seed)`` returns the estimator of Eq. 2
over a fixed sample set as a scalar tensor whose gradient with respect to the
layout ``xy`` (float64 CUDA tensor [n_nodes, 4]) comes from the library's
hand-written backward kernel. The graph object only holds the path data; the
layout passed in is the one differentiated. The graph's own stored layout is
left as it was: forward and backward load ``xy`` into the graph for their
kernels and put the previous layout back afterwards.
"""
from __future__ import annotations

import torch


class _Borrowed:
    """Load xy into the graph for one kernel call, then restore the graph's
    previous layout (an exact round trip: get_coords returns anchor + offset
    in float64, and set_coords re-splits it without rounding)."""

    def __init__(self, graph, xy):
        self.graph, self.xy = graph, xy

    def __enter__(self):
        from . import PgsgdError
        self.saved = torch.empty((self.graph.n_nodes, 4), dtype=torch.float64, device=self.xy.device)
        try:
            self.graph.get_coords(self.saved)
        except PgsgdError:  # the graph holds no layout yet: nothing to restore
            self.saved = None
        self.graph.set_coords(self.xy)
        return self.graph

    def __exit__(self, *exc):
        if self.saved is not None:
            self.graph.set_coords(self.saved)


class SampledStress(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xy, graph, n_pairs, seed):
        with _Borrowed(graph, xy.detach()):
            value, n_valid = graph.dstress(n_pairs, seed)
        ctx.graph = graph
        ctx.n_pairs = n_pairs
        ctx.seed = seed
        ctx.n_valid = n_valid
        ctx.save_for_backward(xy.detach())
        return torch.tensor(value, dtype=torch.float64, device=xy.device)

    @staticmethod
    def backward(ctx, gout):
        (xy,) = ctx.saved_tensors
        graph = ctx.graph
        grad = torch.empty(xy.shape, dtype=torch.float32, device=xy.device)
        scale = float(gout) / max(ctx.n_valid, 1)
        with _Borrowed(graph, xy):
            graph.dstress_backward(ctx.n_pairs, ctx.seed, scale, grad)
        return grad.to(torch.float64), None, None, None


def sampled_stress(xy, graph, n_pairs=10_000_000, seed=1):
    return SampledStress.apply(xy, graph, n_pairs, seed)


def refine(graph, xy, steps=200, lr=0.05, n_pairs=10_000_000, seed=1, resample=False):
    """Gradient refinement of a layout with Adam on the differentiable sampled
    stress. Full batch (default): the same n_pairs pairs every step (seed);
    resample=True draws a fresh set each step (seed + step), a stochastic
    variant. Returns the refined layout and the objective's value per step."""
    x = xy.detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([x], lr=lr)
    trace = []
    for k in range(steps):
        opt.zero_grad()
        f = sampled_stress(x, graph, n_pairs, seed + k if resample else seed)
        f.backward()
        opt.step()
        trace.append(float(f.detach()))
    return x.detach(), trace
