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
