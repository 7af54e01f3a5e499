"""oz2_gemm_noalloc: the emulated DGEMM for callers that cannot have device
memory allocated on their behalf (an application whose own pool owns all
device memory under a hard budget, or a latency-critical loop that cannot take
cudaMalloc's device-wide synchronisation) and cannot pass a workspace either.
It works in the library's fixed device scratch array instead.

Checked through the C ABI against oz2_gemm_ex, on two calls in a row with
different problems (the second call must not see the first call's leftovers in
the shared scratch), and for the size limit.  This file is collected last so a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import paper_pair

pytestmark = pytest.mark.gpu

ULP_TOL = 2   # same tolerance as the parity tests; bit-identical results are expected


def _ulps(a, b):
    ia = np.asarray(a, np.float64).view(np.int64)
    ib = np.asarray(b, np.float64).view(np.int64)
    mask = np.int64(0x7FFFFFFFFFFFFFFF)
    oa = np.where(ia >= 0, ia, -(ia & mask))
    ob = np.where(ib >= 0, ib, -(ib & mask))
    return np.abs(oa - ob)


def test_noalloc_matches_gemm_ex_twice():
    import torch
    from paper_2602_02549_b300 import binding as B
    from paper_2602_02549_b300.build import build
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build()
    cases = [((300, 200, 700), 14, 0.0, 1), ((257, 129, 1030), 0, 1e-15, 2)]
    for (m, n, k), N, tau, seed in cases:
        A, Bm = paper_pair(m, n, k, 1.0, seed=seed)
        At = torch.tensor(A, device="cuda")
        Bt = torch.tensor(Bm, device="cuda")
        C_ref = torch.empty((m, n), dtype=torch.float64, device="cuda")
        C_new = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        assert B.gemm_ex(At, Bt, C_ref, N, 0, target=tau, nmax=20 if N == 0 else 0) == 0
        assert B.gemm_noalloc(At, Bt, C_new, N, 0, target=tau) == 0
        torch.cuda.synchronize()
        assert B.sync() == 0
        assert _ulps(C_new.cpu().numpy(), C_ref.cpu().numpy()).max() <= ULP_TOL


def test_noalloc_rejects_oversize():
    import torch
    from paper_2602_02549_b300 import binding as B
    m = n = k = 1024          # workspace at N = 20 is ~100 MiB > 32 MiB scratch
    A = torch.ones((m, k), dtype=torch.float64, device="cuda")
    Bt = torch.ones((k, n), dtype=torch.float64, device="cuda")
    C = torch.full((m, n), 7.0, dtype=torch.float64, device="cuda")
    assert B.gemm_noalloc(A, Bt, C, 20, 0) == B.OZ2_ENOMEM
    torch.cuda.synchronize()
    assert (C == 7.0).all()   # untouched
