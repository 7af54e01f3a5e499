"""Differentiable emulated GEMM: C = A @ B through the Ozaki-II path, with a
hand-written backward that computes both gradients through the same path.

    dA = dC B^T   (oz2 with OZ2_TRANS_B: B is passed as stored, k x n)
    dB = A^T dC   (oz2 with OZ2_TRANS_A: A is passed as stored, m x k)

Each of the three products picks its own mu, nu and (with nmoduli = 0) its own
N from the bound rule, so every product meets the stated target.  No transposed
copies are made; only a non-row-major gradient is made contiguous first.  In
FP64, when both gradients are wanted, the two backward products go out as one
two-problem oz2_gemm_batched call (one launch per phase for both; each result is
bit-identical to its own oz2_gemm_ex call).
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
        m, k, n = A.size(0), A.size(1), B.size(1)
        if (ctx.needs_input_grad[0] and ctx.needs_input_grad[1] and A.dtype == torch.float64
                and min(m, n, k) > 0 and max(m, n) <= binding.K_MAX):
            dA = torch.empty((m, k), dtype=A.dtype, device=A.device)
            dB = torch.empty((k, n), dtype=A.dtype, device=A.device)
            cfg = dict(nmoduli=ctx.nmoduli, target=ctx.cfg["target"] if ctx.nmoduli == 0 else 0.0,
                       nmax=ctx.cfg["nmax"], fast=ctx.cfg["fast"])
            rc = binding.gemm_batched([dict(A=dC, B=B, C=dA, trans_b=True, **cfg),
                                       dict(A=A, B=dC, C=dB, trans_a=True, **cfg)])
            if rc:
                raise binding.Oz2Error(rc, "oz2_gemm_batched")
            return dA, dB, None, None, None, None
        if ctx.needs_input_grad[0]:
            dA = binding.matmul(dC, B, ctx.nmoduli, trans_b=True, **ctx.cfg)
        if ctx.needs_input_grad[1]:
            dB = binding.matmul(A, dC, ctx.nmoduli, trans_a=True, **ctx.cfg)
        return dA, dB, None, None, None, None


def oz2_matmul(A, B, nmoduli: int = 0, target: float = 1e-15, nmax: int = 0, fast: bool = False):
    """A @ B through the emulation, differentiable in A and B."""
    return Oz2Matmul.apply(A, B, nmoduli, target, nmax, fast)
