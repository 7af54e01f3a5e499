"""Differentiable emulated GEMM: C = A @ B through the Ozaki-II path, with a
hand-written backward that computes both gradients through the same path.

    dA = dC B^T   (oz2 with OZ2_TRANS_B: B is passed as stored, k x n)
    dB = A^T dC   (oz2 with OZ2_TRANS_A: A is passed as stored, m x k)

Each of the three products picks its own mu, nu and (with nmoduli = 0) its own
N from the bound rule, so every product meets the stated target.  No transposed
copies are made; only a non-row-major gradient is made contiguous first.
"""
from __future__ import annotations

import torch

from . import binding


class Oz2Matmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, nmoduli: int = 0, target: float = 1e-15, nmax: int = 0, fast: bool = False):
        ctx.save_for_backward(A, B)
        ctx.cfg = dict(target=target, nmax=nmax, fast=fast)
        ctx.nmoduli = nmoduli
        return binding.matmul(A, B, nmoduli, **ctx.cfg)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        if dC.stride(-1) != 1:
            dC = dC.contiguous()
        dA = dB = None
        if ctx.needs_input_grad[0]:
            dA = binding.matmul(dC, B, ctx.nmoduli, trans_b=True, **ctx.cfg)
        if ctx.needs_input_grad[1]:
            dB = binding.matmul(A, dC, ctx.nmoduli, trans_a=True, **ctx.cfg)
        return dA, dB, None, None, None, None


def oz2_matmul(A, B, nmoduli: int = 0, target: float = 1e-15, nmax: int = 0, fast: bool = False):
    """A @ B through the emulation, differentiable in A and B."""
    return Oz2Matmul.apply(A, B, nmoduli, target, nmax, fast)
