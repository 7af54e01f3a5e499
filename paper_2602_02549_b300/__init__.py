"""B300-native Ozaki-II emulated GEMM (arXiv 2602.02549).

The computation lives in liboz2.so (C ABI, include/oz2.h, CUDA for sm_103a);
`binding` marshals torch tensors into it and `inputs` draws the paper's
synthetic test matrices.
"""
from .binding import Oz2Error, gemm_ex, matmul, sync, workspace_size  # noqa: F401

__all__ = ["Oz2Error", "matmul", "gemm_ex", "workspace_size", "sync"]
