"""Reverse-mode differentiation through the double FFT filter (arXiv:2305.01537, Sec. II.C).

The filter F is linear, so its vector-Jacobian product is the transpose F^T: the phi pass followed
by the theta pass (sph_filter_apply_adjoint). For a chain x_1 = F x_0, x_{k+1} = F(tanh(x_k)) the
library fuses the pointwise map into the filter kernels: the forward step computes F(tanh(z)) and
the backward step (1 - tanh(z)^2) * F^T(g) in one launch each. All arithmetic runs in the CUDA
library; this module only connects it to torch.autograd.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint


class SphFilter(torch.autograd.Function):
    """y = F x; dL/dx = F^T dL/dy."""

    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.apply(x.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.apply_adjoint(g.contiguous()), None


class SphFilterTanh(torch.autograd.Function):
    """y = F(tanh(z)); dL/dz = (1 - tanh(z)^2) * F^T dL/dy (fused)."""

    @staticmethod
    def forward(ctx, z, plan):
        z = z.contiguous()
        ctx.plan = plan
        ctx.save_for_backward(z)
        return plan.apply_tanh(z)

    @staticmethod
    def backward(ctx, g):
        (z,) = ctx.saved_tensors
        return ctx.plan.apply_adjoint_tanh(g.contiguous(), z), None


def sph_filter(x, plan):
    return SphFilter.apply(x, plan)


def sph_filter_tanh(z, plan):
    return SphFilterTanh.apply(z, plan)


def filter_chain(x, plan, n_filters: int = 8, checkpoint_every: int = 0):
    """F_n o tanh o ... o tanh o F_1 applied to x (n filters, n - 1 tanh maps between them).

    checkpoint_every > 0 groups that many steps into a segment whose activations are recomputed
    in the backward pass instead of being kept (only segment inputs are stored)."""
    if n_filters < 1:
        raise ValueError("n_filters must be >= 1")

    def step(k, t):
        return sph_filter(t, plan) if k == 0 else sph_filter_tanh(t, plan)

    if checkpoint_every <= 0:
        y = x
        for k in range(n_filters):
            y = step(k, y)
        return y

    def segment(k0, k1):
        def run(t):
            for k in range(k0, k1):
                t = step(k, t)
            return t
        return run

    y = x
    for k0 in range(0, n_filters, checkpoint_every):
        k1 = min(n_filters, k0 + checkpoint_every)
        y = checkpoint(segment(k0, k1), y, use_reentrant=False)
    return y


def chain_loss(x, plan, w, n_filters: int = 8, checkpoint_every: int = 0):
    """sum(w * y^2) with y the filter chain of x."""
    y = filter_chain(x, plan, n_filters, checkpoint_every)
    return (w * y * y).sum()
