"""Parity on problems with more than two waves of output tiles and k >= 2048,
the regime of the longest residue GEMMs:

* a single call with 333 tiles of 128 x 256 (two full waves of 148 and a
  partial one): sampled entries recomputed by the oracle with the GPU's
  exponents, bit for bit, and the W_l of sampled rows and columns equal the
  oracle's, for a fixed N and the bound rule;
* problems with k >= 2048 inside a batch equal the same problems as single
  calls, bit for bit;
* an SGEMM single call of 320 tiles, sampled entries bit for bit.
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


@pytest.mark.parametrize("N", [14, 0])
def test_single_call_many_waves(oracle, N):
    import torch
    from paper_2602_02549_b300 import binding as B
    # 37 x 9 = 333 tiles of 128 x 256 (148 SMs: two full waves and a partial one of 37)
    m, n, k = 128 * 37 - 5, 256 * 8 + 100, 2100
    A, Bm = paper_pair(m, n, k, 1.0, seed=5)
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(Bm, device="cuda")
    nplanes = N or 20
    mu = torch.empty(m, dtype=torch.int32, device="cuda")
    nu = torch.empty(n, dtype=torch.int32, device="cuda")
    nout = torch.zeros(1, dtype=torch.int32, device="cuda")
    W = torch.zeros(nplanes * m * n, dtype=torch.int8, device="cuda")
    C = B.matmul(At, Bt, N, target=1e-15, nmax=20, mu_out=mu, nu_out=nu, n_out=nout, w_out=W)
    torch.cuda.synchronize()
    assert B.sync() == 0
    Nu = int(nout.item())
    rng = np.random.default_rng(7)
    # rows and columns from the first tiles of the raster and from the last ones
    ii = np.unique(np.concatenate([[0, m - 1, m - 130], rng.integers(0, m, 20)]))
    jj = np.unique(np.concatenate([[0, n - 1, n - 257], rng.integers(0, n, 20)]))
    A_rows, B_cols = np.ascontiguousarray(A[ii]), np.ascontiguousarray(Bm[:, jj])
    mu_s, nu_s = mu.cpu().numpy()[ii], nu.cpu().numpy()[jj]
    ref = oracle.os_ii_block(A_rows, B_cols, mu_s, nu_s, Nu)
    got = C.cpu().numpy()[np.ix_(ii, jj)]
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    Ap = oracle.trunc_scaled_rows(A_rows, mu_s)
    Bp = np.ascontiguousarray(oracle.trunc_scaled_rows(B_cols.T, nu_s).T)
    Wref = oracle.crt(Ap, Bp, Nu)["W"]
    Wg = W.cpu().numpy().reshape(nplanes, m, n)[:Nu][:, ii][:, :, jj]
    assert np.array_equal(Wg, Wref)


def test_long_k_batch_equals_single_calls():
    import torch
    from paper_2602_02549_b300 import binding as B
    shapes = [(300, 500, 2500, 1.0), (1000, 700, 3000, 2.0), (200, 300, 400, 0.5), (130, 260, 4097, 4.0)]
    probs, singles = [], []
    for i, (m, n, k, phi) in enumerate(shapes):
        A, Bm = paper_pair(m, n, k, phi, seed=60 + i)
        At, Bt = torch.tensor(A, device="cuda"), torch.tensor(Bm, device="cuda")
        probs.append(dict(A=At, B=Bt, C=torch.empty((m, n), dtype=torch.float64, device="cuda"), nmoduli=0,
                          target=1e-14, nmax=20, n_out=torch.zeros(1, dtype=torch.int32, device="cuda")))
        singles.append(B.matmul(At, Bt, 0, target=1e-14, nmax=20))
    assert B.gemm_batched(probs) == 0
    torch.cuda.synchronize()
    assert B.sync() == 0
    for q, ref in zip(probs, singles):
        assert torch.equal(q["C"], ref)


def test_sgemm_many_waves(oracle):
    import torch
    from paper_2602_02549_b300 import binding as B
    m, n, k = 128 * 40, 256 * 8, 2048
    A, Bm = paper_pair(m, n, k, 1.0, seed=9, dtype=np.float32)
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(Bm, device="cuda")
    mu = torch.empty(m, dtype=torch.int32, device="cuda")
    nu = torch.empty(n, dtype=torch.int32, device="cuda")
    C = B.matmul(At, Bt, 9, mu_out=mu, nu_out=nu)
    torch.cuda.synchronize()
    assert B.sync() == 0
    rng = np.random.default_rng(3)
    ii = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m, 16)]))
    jj = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 16)]))
    A_rows = np.ascontiguousarray(A[ii].astype(np.float64))
    B_cols = np.ascontiguousarray(Bm[:, jj].astype(np.float64))
    ref = oracle.os_ii_block(A_rows, B_cols, mu.cpu().numpy()[ii], nu.cpu().numpy()[jj], 9, 32)
    got = C.cpu().numpy()[np.ix_(ii, jj)]
    assert np.array_equal(got.view(np.int32), ref.view(np.int32))
