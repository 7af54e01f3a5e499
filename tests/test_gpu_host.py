"""Host-array entry points (oz2_gemm_host, oz2_sgemm_host): the library copies
A and B to the device, runs the emulation and copies C back on the caller's
stream.  Every result must be bit-identical to oz2_gemm_ex / oz2_sgemm_ex on
device copies of the same operands (whose parity with the oracle the other
tests check): pinned and pageable host memory, leading dimensions wider than
the rows, transposes, FP32, the bound rule, and two streams with two
workspaces alternating as the benchmark's end-to-end pipeline runs them."""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import paper_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2602_02549_b300.build import build
    build()


def _device_reference(A, Bm, N, mode, target, nmax):
    import torch
    from paper_2602_02549_b300 import binding as B
    dA, dB = A.cuda(), Bm.cuda()
    ta, tb = bool(mode & B.OZ2_TRANS_A), bool(mode & B.OZ2_TRANS_B)
    m = A.size(1) if ta else A.size(0)
    n = Bm.size(0) if tb else Bm.size(1)
    C = torch.empty((m, n), dtype=A.dtype, device="cuda")
    nout = torch.zeros(8, dtype=torch.int32, device="cuda")     # one N per K range (k <= 8 2^17)
    assert B.gemm_ex(dA.contiguous(), dB.contiguous(), C, N, mode, target=target, nmax=nmax, n_out=nout) == 0
    torch.cuda.synchronize()
    return C.cpu(), int(nout[0].item())


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("m,n,k,ta,tb,N", [(300, 200, 150, False, False, 14), (129, 257, 1000, True, False, 0),
                                           (1, 3, 5, False, True, 8), (64, 65, 66, True, True, 0)])
def test_host_arrays_equal_device_call(pinned, fp32, m, n, k, ta, tb, N):
    import torch
    from paper_2602_02549_b300 import binding as B
    dt = torch.float32 if fp32 else torch.float64
    A = paper_matrix(m, k, 1.0, 1)
    Bm = paper_matrix(k, n, 1.0, 2)
    As = torch.tensor(np.ascontiguousarray(A.T) if ta else A, dtype=dt)
    Bs = torch.tensor(np.ascontiguousarray(Bm.T) if tb else Bm, dtype=dt)
    if pinned:
        As, Bs = As.pin_memory(), Bs.pin_memory()
    C = torch.full((m, n), float("nan"), dtype=dt)
    if pinned:
        C = C.pin_memory()
    mode = (B.OZ2_TRANS_A if ta else 0) | (B.OZ2_TRANS_B if tb else 0)
    target = (1e-7 if fp32 else 1e-15) if N == 0 else 0.0
    nmax = (14 if fp32 else 20) if N == 0 else 0
    nout = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert B.gemm_host(As, Bs, C, N, mode, target=target, nmax=nmax, n_out=nout) == 0
    assert B.sync() == 0
    ref, nref = _device_reference(As, Bs, N, mode, target, nmax)
    assert int(nout.item()) == nref
    assert torch.equal(C, ref)


def test_host_strided_views():
    # host views into wider arrays: lda, ldb, ldc beyond the row lengths
    import torch
    from paper_2602_02549_b300 import binding as B
    m, n, k = 77, 45, 300
    Aw = torch.tensor(paper_matrix(m, k + 13, 1.0, 5)).pin_memory()
    Bw = torch.tensor(paper_matrix(k, n + 7, 1.0, 6)).pin_memory()
    Cw = torch.full((m, n + 3), 7.0, dtype=torch.float64).pin_memory()
    A, Bv, C = Aw[:, :k], Bw[:, :n], Cw[:, :n]
    assert B.gemm_host(A, Bv, C, 16, 0) == 0
    assert B.sync() == 0
    ref, _ = _device_reference(A.contiguous(), Bv.contiguous(), 16, 0, 0.0, 0)
    assert torch.equal(C, ref)
    assert (Cw[:, n:] == 7.0).all()            # columns past n untouched


def test_two_streams_two_workspaces():
    # alternating calls on two streams, each with its own workspace and pinned
    # buffers: every result equals the device call's
    import torch
    from paper_2602_02549_b300 import binding as B
    m = n = k = 512
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ws = [torch.empty(B.host_workspace_size(m, n, k, 20), dtype=torch.uint8, device="cuda") for _ in range(2)]
    As = [torch.tensor(paper_matrix(m, k, 1.0, 10 + s)).pin_memory() for s in range(6)]
    Bs = [torch.tensor(paper_matrix(k, n, 1.0, 20 + s)).pin_memory() for s in range(6)]
    Cs = [torch.empty((m, n), dtype=torch.float64).pin_memory() for _ in range(6)]
    for s in range(6):
        assert B.gemm_host(As[s], Bs[s], Cs[s], 0, 0, target=1e-15, nmax=20, workspace=ws[s % 2],
                           stream=streams[s % 2]) == 0
    torch.cuda.synchronize()
    assert B.sync() == 0
    for s in range(6):
        ref, _ = _device_reference(As[s], Bs[s], 0, 0, 1e-15, 20)
        assert torch.equal(Cs[s], ref)


def test_host_workspace_too_small():
    import torch
    from paper_2602_02549_b300 import binding as B
    A = torch.tensor(paper_matrix(40, 30, 1.0, 1))
    Bm = torch.tensor(paper_matrix(30, 20, 1.0, 2))
    C = torch.empty((40, 20), dtype=torch.float64)
    small = torch.empty(B.host_workspace_size(40, 20, 30, 14) - 256, dtype=torch.uint8, device="cuda")
    before = B.launch_count()
    assert B.gemm_host(A, Bm, C, 14, 0, workspace=small) == B.OZ2_ENOMEM
    assert B.launch_count() == before


def test_host_arrays_split_k():
    # k beyond 2^17: the ranges run in the emulation's workspace after the
    # uploads, as in the device call
    import torch
    from paper_2602_02549_b300 import binding as B
    m, n, k = 9, 7, (1 << 17) + 100
    A = torch.tensor(paper_matrix(m, k, 1.0, 41)).pin_memory()
    Bm = torch.tensor(paper_matrix(k, n, 1.0, 42)).pin_memory()
    C = torch.empty((m, n), dtype=torch.float64).pin_memory()
    assert B.gemm_host(A, Bm, C, 0, 0, target=1e-15, nmax=20) == 0
    assert B.sync() == 0
    ref, _ = _device_reference(A, Bm, 0, 0, 1e-15, 20)
    assert torch.equal(C, ref)
