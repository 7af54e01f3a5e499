"""Leading dimensions larger than the rows: A, B and C given as column slices of
wider arrays (lda, ldb, ldc above k or n, odd pads, so that rows start off the
16-byte boundary the kernels' vector loads take when they can).  The result
must be bit-identical to the same call on contiguous copies, and C's pad
columns must be left as they were.
"""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import paper_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2602_02549_b300.build import build
    build()


def _padded(x, pad, dev, dt):
    """x as a column slice of a (rows, cols + pad) device array filled with NaN."""
    import torch
    big = torch.full((x.shape[0], x.shape[1] + pad), float("nan"), dtype=dt, device=dev)
    big[:, : x.shape[1]] = torch.tensor(x, dtype=dt, device=dev)
    return big[:, : x.shape[1]]


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("nmoduli", [0, 9])
def test_leading_dimensions(fp32, ta, tb, nmoduli):
    import torch
    from paper_2602_02549_b300 import binding as B

    m, n, k = 150, 200, 700
    dt = torch.float32 if fp32 else torch.float64
    A, Bm = paper_pair(m, n, k, 1.0, seed=11, dtype=np.float32 if fp32 else np.float64)
    As = np.ascontiguousarray(A.T) if ta else A
    Bs = np.ascontiguousarray(Bm.T) if tb else Bm
    mode = (B.OZ2_TRANS_A if ta else 0) | (B.OZ2_TRANS_B if tb else 0)
    target = 0.0 if nmoduli else (1e-7 if fp32 else 1e-15)

    Ac = torch.tensor(As, dtype=dt, device="cuda")
    Bc = torch.tensor(Bs, dtype=dt, device="cuda")
    Cc = torch.empty((m, n), dtype=dt, device="cuda")
    assert B.gemm_ex(Ac, Bc, Cc, nmoduli, mode, target=target, nmax=20) == 0

    Av, Bv = _padded(As, 3, "cuda", dt), _padded(Bs, 5, "cuda", dt)
    Cbig = torch.full((m, n + 7), -1.5, dtype=dt, device="cuda")
    Cv = Cbig[:, :n]
    assert Av.stride(0) > Av.size(1) and Bv.stride(0) > Bv.size(1) and Cv.stride(0) == n + 7
    assert B.gemm_ex(Av, Bv, Cv, nmoduli, mode, target=target, nmax=20) == 0
    torch.cuda.synchronize()
    assert B.sync() == 0

    got, ref = Cv.cpu().numpy(), Cc.cpu().numpy()
    ib = np.int32 if fp32 else np.int64
    assert np.array_equal(got.view(ib), ref.view(ib))
    assert bool((Cbig[:, n:] == -1.5).all())
