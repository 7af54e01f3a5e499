"""Parity at the benchmark's full size: DGEMM 16384^3, phi = 1, the bound rule
with tau = 1e-15 and nmax = 20, called exactly as bench.py calls it (one
oz2_gemm_ex with a caller workspace on the current stream).

The oracle cannot redo the whole product, so the test checks what it can
compute entry by entry or row by row:
  * sampled entries C_ij (a block of rows x columns that includes the first and
    last row and column) recomputed by the oracle with the GPU's mu, nu and N
    (Algorithm 2 leaves each entry a function of row i of A and column j of B
    once the exponents are fixed): within ULP_TOL (0 expected);
  * Theorem 2's bound on those entries, against the exact products;
  * mu_i and nu_j of sampled rows and columns inside the band Algorithm 2
    allows, from the oracle's own Abar, Bbar and the exact row/column maxima of
    Cbar = Abar Bbar.
"""
import numpy as np
import pytest

from _gpu_util import ulp_distance

pytestmark = pytest.mark.gpu

SIZE = 16384
ULP_TOL = 2


@pytest.fixture(scope="module")
def fullsize():
    import torch
    from paper_2602_02549_b300 import binding as B
    from paper_2602_02549_b300.build import build
    from paper_2602_02549_b300.inputs import paper_matrix_torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build()
    dev = torch.device("cuda", 0)
    m = n = k = SIZE
    A = paper_matrix_torch(m, k, 1.0, 0, dev)
    Bm = paper_matrix_torch(k, n, 1.0, 1, dev)
    C = torch.empty((m, n), dtype=torch.float64, device=dev)
    ws = torch.empty(B.workspace_size(m, n, k, 20, 0, False), dtype=torch.uint8, device=dev)
    nout = torch.zeros(1, dtype=torch.int32, device=dev)
    mu = torch.empty(m, dtype=torch.int32, device=dev)
    nu = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rc = B.gemm_ex(A, Bm, C, 0, 0, target=1e-15, nmax=20, workspace=ws, stream=stream, n_out=nout,
                   mu_out=mu, nu_out=nu)
    assert rc == 0
    torch.cuda.synchronize()
    assert B.sync(stream) == 0
    out = dict(A=A.cpu().numpy(), B=Bm.cpu().numpy(), C=C.cpu().numpy(), mu=mu.cpu().numpy(),
               nu=nu.cpu().numpy(), N=int(nout.item()))
    del ws, C, A, Bm
    torch.cuda.empty_cache()
    return out


def _sample(rng, size, count):
    idx = rng.choice(np.arange(1, size - 1), size=count - 2, replace=False)
    return np.sort(np.concatenate([[0, size - 1], idx]))


def test_fullsize_sampled_entries(oracle, fullsize):
    f = fullsize
    assert 2 <= f["N"] <= 20
    rng = np.random.default_rng(2024)
    ii = _sample(rng, SIZE, 24)
    jj = _sample(rng, SIZE, 24)
    A_rows = np.ascontiguousarray(f["A"][ii])
    B_cols = np.ascontiguousarray(f["B"][:, jj])
    mu, nu, N = f["mu"][ii], f["nu"][jj], f["N"]
    ref = oracle.os_ii_block(A_rows, B_cols, mu, nu, N)
    got = f["C"][np.ix_(ii, jj)]
    assert ulp_distance(got, ref).max() <= ULP_TOL
    # Theorem 2 on the sampled entries (the exponents the GPU used)
    Ap = oracle.trunc_scaled_rows(A_rows, mu)
    Bp = np.ascontiguousarray(oracle.trunc_scaled_rows(B_cols.T, nu).T)
    assert oracle.lemma0_holds(Ap, Bp, N)
    eb = oracle.bound_from_exponents(A_rows, B_cols, mu, nu, Ap, Bp, N) + 2.0 ** -1075
    err = np.abs(oracle.exact_residual(A_rows, B_cols, got))
    assert (err <= eb).all()


def test_fullsize_exponents_in_band(oracle, fullsize):
    # Abar, Bbar as Algorithm 2 defines them (oracle), then the exact maxima of
    # Cbar over whole rows / columns for the sampled indices (integer sums below
    # 2^26, exact in FP64)
    f = fullsize
    rng = np.random.default_rng(7)
    ii = _sample(rng, SIZE, 6)
    jj = _sample(rng, SIZE, 6)
    s_row = oracle.scaling(np.ascontiguousarray(f["A"][ii]), f["B"][:, :1], f["N"])
    s_col = oracle.scaling(f["A"][:1], np.ascontiguousarray(f["B"][:, jj]), f["N"])
    # full Abar and Bbar are needed for the maxima over all columns / rows
    alpha = oracle.floor_log2_absmax(f["A"], axis=1)
    beta = oracle.floor_log2_absmax(f["B"], axis=0)
    assert np.array_equal(s_row["alpha"], alpha[ii]) and np.array_equal(s_col["beta"], beta[jj])
    Abar_rows = s_row["Abar"].astype(np.float64)                  # rows ii, all h
    Bbar_cols = s_col["Bbar"].astype(np.float64)                  # all h, columns jj
    Bbar = _bbar_full(oracle, f["B"], beta).astype(np.float64)   # all h, all j
    Abar = _abar_full(oracle, f["A"], alpha).astype(np.float64)  # all i, all h
    cmax_row = (Abar_rows @ Bbar).max(axis=1)
    cmax_col = (Abar @ Bbar_cols).max(axis=0)
    lo, hi = oracle.mu_band(s_row["mu_p"], cmax_row, f["N"])
    assert ((f["mu"][ii] >= lo) & (f["mu"][ii] <= hi)).all()
    lo, hi = oracle.mu_band(s_col["nu_p"], cmax_col, f["N"])
    assert ((f["nu"][jj] >= lo) & (f["nu"][jj] <= hi)).all()


def _abar_full(oracle, A, alpha):
    mu_p = np.where(alpha == oracle.INT32_MIN, 0, 5 - alpha.astype(np.int64)).astype(np.int32)
    out = np.empty(A.shape, dtype=np.int8)
    rs, cs = oracle._strides(A)
    oracle.lib().oz2o_ceil_scaled_abs(A.shape[0], A.shape[1], oracle._p(A), rs, cs, oracle._p(mu_p),
                                      oracle._p(out))
    return out


def _bbar_full(oracle, B, beta):
    return np.ascontiguousarray(_abar_full(oracle, np.ascontiguousarray(B.T), beta).T)


def test_fullsize_sgemm_sampled_entries(oracle):
    # the SGEMM benchmark's call: 8192^3 FP32, phi = 1, bound rule tau = 1e-7, nmax = 14
    import torch
    from paper_2602_02549_b300 import binding as B
    from paper_2602_02549_b300.inputs import paper_matrix_torch
    dev = torch.device("cuda", 0)
    s = 8192
    A = paper_matrix_torch(s, s, 1.0, 0, dev, torch.float32)
    Bm = paper_matrix_torch(s, s, 1.0, 1, dev, torch.float32)
    C = torch.empty((s, s), dtype=torch.float32, device=dev)
    nout = torch.zeros(1, dtype=torch.int32, device=dev)
    mu = torch.empty(s, dtype=torch.int32, device=dev)
    nu = torch.empty(s, dtype=torch.int32, device=dev)
    ws = torch.empty(B.workspace_size(s, s, s, 14, 0, True), dtype=torch.uint8, device=dev)
    assert B.gemm_ex(A, Bm, C, 0, 0, target=1e-7, nmax=14, workspace=ws, n_out=nout, mu_out=mu, nu_out=nu) == 0
    torch.cuda.synchronize()
    assert B.sync() == 0
    N = int(nout.item())
    rng = np.random.default_rng(5)
    ii = _sample(rng, s, 24)
    jj = _sample(rng, s, 24)
    A_rows = A[ii].double().cpu().numpy()
    B_cols = Bm[:, jj].double().cpu().numpy()
    mu_s, nu_s = mu.cpu().numpy()[ii], nu.cpu().numpy()[jj]
    ref = oracle.os_ii_block(A_rows, B_cols, mu_s, nu_s, N, 32)
    got = C.cpu().numpy()[np.ix_(ii, jj)].astype(np.float64)
    assert ulp_distance(got, ref, fp32=True).max() <= ULP_TOL
    Ap = oracle.trunc_scaled_rows(A_rows, mu_s)
    Bp = np.ascontiguousarray(oracle.trunc_scaled_rows(B_cols.T, nu_s).T)
    eb = oracle.bound_from_exponents(A_rows, B_cols, mu_s, nu_s, Ap, Bp, N, 32) + 2.0 ** -150
    assert (np.abs(oracle.exact_residual(A_rows, B_cols, got)) <= eb).all()
