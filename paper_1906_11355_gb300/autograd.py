"""Differentiable MCLAHE: a torch.autograd.Function over the C ABI.

The forward pass is mclahe_forward; the backward pass is mclahe_backward,
which returns dL/dclip_limit through the clip/redistribute, cumulative-sum and
normalisation steps of Algorithm 1 (arXiv:1906.11355).  The output is
piecewise constant in the intensities, so the input gradient is zero almost
everywhere and is returned as zeros.  PyTorch supplies memory and streams;
every step runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import _native as nat
from .api import MCLAHE


class MCLAHEFunction(torch.autograd.Function):
    """out = MCLAHE(x; clip) for one volume.  clip: 1-element float32 CUDA
    tensor (the clip limit, read on the device); op: an api.MCLAHE holding the
    plan.  Each forward call keeps its own workspace (range, histograms and
    tables) for the backward call."""

    @staticmethod
    def forward(ctx, x, clip, op):
        op._check_volume(x)
        clip = clip.reshape(1).contiguous()
        ws = torch.zeros(op.ws_bytes, dtype=torch.uint8, device=x.device)
        out = torch.empty_like(x)
        nat.mclahe_forward(op.plan, x, out, ws, op.ws_bytes, clip)
        ctx.save_for_backward(x, clip)
        ctx.ws = ws
        ctx.op = op
        return out

    @staticmethod
    def backward(ctx, grad_out):
        x, clip = ctx.saved_tensors
        op = ctx.op
        grad_clip = torch.empty(1, dtype=torch.float32, device=x.device)
        nat.mclahe_backward(op.plan, x, grad_out.contiguous(), ctx.ws, op.ws_bytes, clip, None,
                            grad_clip)
        gx = torch.zeros_like(x) if ctx.needs_input_grad[0] else None
        gc = grad_clip.reshape(ctx.saved_tensors[1].shape) if ctx.needs_input_grad[1] else None
        return gx, gc, None


class MCLAHEBatchFunction(torch.autograd.Function):
    """out[b] = MCLAHE(x[b]; clip[b]) for a batch x [B, *shape] of volumes of
    one plan.  The forward pass is one mclahe_forward_batch call (every
    volume's forward on parallel branches, each with its own workspace); the
    backward pass is one mclahe_backward_batch call (three launches per 32
    volumes)."""

    @staticmethod
    def forward(ctx, x, clip, op):
        if x.dim() != len(op.shape) + 1 or tuple(x.shape[1:]) != tuple(op.shape):
            raise ValueError("x must be [B, *shape] of the plan's shape")
        x = x.contiguous()
        clip = clip.reshape(-1).contiguous()
        if clip.numel() != x.shape[0]:
            raise ValueError("one clip limit per volume")
        out = torch.empty_like(x)
        ws = [torch.zeros(op.ws_bytes, dtype=torch.uint8, device=x.device) for _ in range(x.shape[0])]
        nat.mclahe_forward_batch(op.plan, list(x), list(out), ws, op.ws_bytes, clip)
        ctx.save_for_backward(x, clip)
        ctx.ws = ws
        ctx.op = op
        return out

    @staticmethod
    def backward(ctx, grad_out):
        x, clip = ctx.saved_tensors
        op = ctx.op
        g = grad_out.contiguous()
        grad_clip = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        nat.mclahe_backward_batch(op.plan, [x[b] for b in range(x.shape[0])],
                                  [g[b] for b in range(x.shape[0])], ctx.ws, op.ws_bytes, clip, grad_clip)
        gx = torch.zeros_like(x) if ctx.needs_input_grad[0] else None
        return gx, grad_clip if ctx.needs_input_grad[1] else None, None


_ops = {}


def _op(shape, kernel_size, n_bins, adaptive, global_range, device):
    key = (tuple(shape), tuple(int(b) for b in kernel_size), int(n_bins), bool(adaptive),
           None if global_range is None else tuple(float(v) for v in global_range), str(device))
    op = _ops.get(key)
    if op is None:
        op = MCLAHE(shape, kernel_size, n_bins, 0.0, adaptive, global_range, device)
        _ops[key] = op
    return op


def mclahe_autograd(x, clip, kernel_size, n_bins=256, adaptive=False, global_range=None):
    """Differentiable MCLAHE of x ([*shape] or a batch [B, *shape]) with a
    learnable clip limit (a tensor of B values, or one value for one volume).
    Returns the output with the shape of x."""
    nd = len(kernel_size)
    if x.dim() == nd:
        op = _op(x.shape, kernel_size, n_bins, adaptive, global_range, x.device)
        return MCLAHEFunction.apply(x, clip.reshape(1), op)
    if x.dim() != nd + 1:
        raise ValueError("x must have len(kernel_size) or len(kernel_size) + 1 dimensions")
    op = _op(x.shape[1:], kernel_size, n_bins, adaptive, global_range, x.device)
    return MCLAHEBatchFunction.apply(x, clip.reshape(-1), op)
