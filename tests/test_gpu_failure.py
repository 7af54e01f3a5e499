"""Failure detection without a GPU fault: a device wait that gives up reports
OZ2_ETIMEOUT through oz2_sync, the status is then cleared, and the library
(and the CUDA context) keep working."""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import paper_pair

from _gpu_util import run_gpu

pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_recovers():
    import torch
    from paper_2602_02549_b300 import binding as B
    from paper_2602_02549_b300.build import build
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build()
    assert B.wait_selftest(0) == B.OZ2_EINVAL
    assert B.wait_selftest(20000) == 0          # 20 ms, then the wait gives up
    assert B.sync() == B.OZ2_ETIMEOUT
    assert B.sync() == 0                         # the status word was cleared
    A, Bm = paper_pair(64, 80, 300, 1.0, seed=1)
    g = run_gpu(A, Bm, 14)                       # a normal call afterwards
    assert np.isfinite(g["C"]).all()
    assert np.abs(g["C"] - A @ Bm).max() <= 1e-12 * np.abs(A).max() * np.abs(Bm).max() * 300


def test_gemm_wait_expires_drains_and_recovers():
    # the residue GEMM's own failure path: one operand stage armed but never
    # loaded, so the MMA warp's bounded wait gives up; every CTA then waits for
    # the copies and MMAs it had issued, frees its TMEM and returns (no fault,
    # no hang), oz2_sync reports OZ2_ETIMEOUT once, and the next call is exact
    import time
    import torch
    from paper_2602_02549_b300 import binding as B
    m, n, k, N = 300, 520, 1100, 14
    A, Bm = paper_pair(m, n, k, 1.0, seed=4)
    At = torch.tensor(A, device="cuda")
    Bt = torch.tensor(Bm, device="cuda")
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    ref = B.matmul(At, Bt, N)
    torch.cuda.synchronize()
    assert B.sync() == 0
    assert B.gemm_timeout_selftest(At, Bt, C, N, 0) == B.OZ2_EINVAL
    t0 = time.perf_counter()
    assert B.gemm_timeout_selftest(At, Bt, C, N, 5000) == 0      # 5 ms per wait
    assert B.sync() == B.OZ2_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0                          # the waits ended by themselves
    assert B.sync() == 0
    again = B.matmul(At, Bt, N)
    torch.cuda.synchronize()
    assert B.sync() == 0
    assert torch.equal(again, ref)
