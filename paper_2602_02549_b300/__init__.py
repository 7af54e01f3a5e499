"""B300-native Ozaki-II emulated GEMM (arXiv 2602.02549).

The computation lives in liboz2.so (C ABI, include/oz2.h, CUDA for sm_103a);
`binding` marshals torch tensors into it, `autograd` wraps it for
torch.autograd and `inputs` draws the paper's synthetic test matrices.
"""
from .binding import Oz2Error, gemm_ex, matmul, sync, workspace_size  # noqa: F401
from .autograd import Oz2Matmul, oz2_matmul  # noqa: F401

__all__ = ["Oz2Error", "matmul", "gemm_ex", "workspace_size", "sync", "Oz2Matmul", "oz2_matmul"]
