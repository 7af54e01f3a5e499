"""The padded rows of the residue planes (rows m .. m_pad-1 of A'_l, n .. n_pad-1
of B'_l) are not written by the residue kernels: they reach only rows or
columns of C'_l past m or n, which the CRT never reads.  These tests start a
call from a workspace full of NaN bytes, or of large finite BF16 values, and
check that N and every bit of C equal those of a call from a zeroed workspace."""
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


FILLS = (0x00, 0xFF, 0x7F)     # zeros; BF16 0xFFFF (NaN); BF16 0x7F7F (3.4e38)


@pytest.mark.parametrize("m,n,k,trans_b", [(300, 200, 150, False), (129, 257, 1000, True), (1, 3, 5, False)])
def test_single_call_ignores_workspace_contents(m, n, k, trans_b):
    import torch
    from paper_2602_02549_b300 import binding as B
    A = torch.tensor(paper_matrix(m, k, 1.0, 0), device="cuda")
    Bm = paper_matrix(k, n, 1.0, 1)
    Bt = torch.tensor(Bm.T.copy() if trans_b else Bm, device="cuda")
    mode = B.OZ2_TRANS_B if trans_b else 0
    size = B.workspace_size(m, n, k, 20)
    outs = []
    for fill in FILLS:
        ws = torch.full((size,), fill, dtype=torch.uint8, device="cuda")
        C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        nout = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert B.gemm_ex(A, Bt, C, 0, mode, target=1e-15, nmax=20, workspace=ws, n_out=nout) == 0
        torch.cuda.synchronize()
        assert B.sync() == 0
        outs.append((int(nout.item()), C.cpu()))
    for N, C in outs[1:]:
        assert N == outs[0][0]
        assert torch.equal(C, outs[0][1])
    assert not torch.isnan(outs[0][1]).any()


def test_batched_call_ignores_workspace_contents():
    import torch
    from paper_2602_02549_b300 import binding as B
    shapes = [(300, 200, 150), (33, 65, 17), (513, 129, 700), (1, 1, 1), (250, 260, 300)]
    ref = None
    for fill in FILLS:
        probs = []
        for i, (m, n, k) in enumerate(shapes):
            probs.append(dict(A=torch.tensor(paper_matrix(m, k, 1.0, 2 * i), device="cuda"),
                              B=torch.tensor(paper_matrix(k, n, 1.0, 2 * i + 1), device="cuda"),
                              C=torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda"),
                              nmoduli=0, target=1e-14, nmax=30, fast=False,
                              n_out=torch.zeros(1, dtype=torch.int32, device="cuda")))
        ws = torch.full((B.batched_workspace_size(probs),), fill, dtype=torch.uint8, device="cuda")
        assert B.gemm_batched(probs, workspace=ws) == 0
        torch.cuda.synchronize()
        assert B.sync() == 0
        got = [(int(q["n_out"].item()), q["C"].cpu()) for q in probs]
        if ref is None:
            ref = got
            assert all(not torch.isnan(C).any() for _, C in got)
        else:
            for (N0, C0), (N1, C1) in zip(ref, got):
                assert N0 == N1
                assert torch.equal(C0, C1)
