"""Row-sharded calls on one GPU with the ranks emulated one after another: each
rank's oz2_gemm_rows_begin, the exchange done here with torch (element-wise
maximum over the ranks of the three arrays, written back in place, as an
all-reduce would), then each rank's oz2_gemm_rows_end.  The stacked rows of C
and the N equal one unsharded call bit for bit (Algorithm 2's nu_j takes the
column maxima of Cbar over all rows; the bound rule the maxima over all rows).
No kernel waits on another rank: the ranks' launches run one after another."""
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


def run_ranks(At, Bt, m, n, k, N, tau, R, mode, exchange=True):
    import torch
    from paper_2602_02549_b300 import binding as B
    ta = bool(mode & B.OZ2_TRANS_A)
    parts = np.array_split(np.arange(m), R)
    ranks = []
    for rows in parts:
        r0, r1 = int(rows[0]), int(rows[-1]) + 1
        Ar = At[:, r0:r1] if ta else At[r0:r1]
        ws = torch.empty(B.workspace_size(r1 - r0, n, k, N or 20, mode, False), dtype=torch.uint8, device="cuda")
        arrays = B.gemm_rows_begin(Ar, Bt, N, mode, workspace=ws, target=tau, nmax=20)
        ranks.append((Ar, ws, arrays, r1 - r0))
    if exchange:
        for i in range(3):
            mx = ranks[0][2][i].clone()
            for rk in ranks[1:]:
                mx = torch.maximum(mx, rk[2][i])
            for rk in ranks:
                rk[2][i].copy_(mx)
    Cs, Ns = [], []
    for Ar, ws, _, mr in ranks:
        C = torch.empty((mr, n), dtype=torch.float64, device="cuda")
        nout = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert B.gemm_rows_end(Ar, Bt, C, N, mode, workspace=ws, target=tau, nmax=20, n_out=nout) == 0
        Cs.append(C)
        Ns.append(nout)
    torch.cuda.synchronize()
    assert B.sync() == 0
    return torch.cat(Cs), [int(x.item()) for x in Ns]


CASES = [(700, 300, 900, 1.0, 0, 1e-15, 2, 0), (1000, 260, 1500, 4.0, 14, 0.0, 3, 0),
         (333, 200, 400, 2.0, 0, 1e-12, 3, 6), (129, 513, 2000, 0.5, 0, 1e-15, 2, 4), (5, 40, 70, 1.0, 0, 1e-15, 5, 0)]


@pytest.mark.parametrize("case", CASES)
def test_sharded_rows_equal_unsharded(case):
    import torch
    from paper_2602_02549_b300 import binding as B
    m, n, k, phi, N, tau, R, mode = case
    A, Bm = paper_pair(m, n, k, phi, seed=m + R)
    At = torch.tensor(A.T.copy() if mode & B.OZ2_TRANS_A else A, device="cuda")
    Bt = torch.tensor(Bm.T.copy() if mode & B.OZ2_TRANS_B else Bm, device="cuda")
    nref = torch.zeros(1, dtype=torch.int32, device="cuda")
    ref = torch.empty((m, n), dtype=torch.float64, device="cuda")
    assert B.gemm_ex(At, Bt, ref, N, mode, target=tau, nmax=20, n_out=nref) == 0
    C, Ns = run_ranks(At, Bt, m, n, k, N, tau, R, mode)
    assert torch.equal(C, ref)
    assert Ns == [int(nref.item())] * R


def test_exchange_is_needed():
    # without the exchange each rank scales its B columns by its own rows' Cbar
    # maxima: a valid emulation, but not the unsharded one
    import torch
    from paper_2602_02549_b300 import binding as B
    m, n, k = 600, 300, 800
    A, Bm = paper_pair(m, n, k, 4.0, seed=3)
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(Bm, device="cuda")
    ref = B.matmul(At, Bt, 14)
    C, _ = run_ranks(At, Bt, m, n, k, 14, 0.0, 2, 0, exchange=False)
    assert not torch.equal(C, ref)
