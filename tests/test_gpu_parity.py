"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bars (the tolerances are written in each test):
  * W_l = mod(A'_l B'_l, p_l): bit-exact (integer work);
  * mu, nu: inside the band Algorithm 2 allows under assumption (1) on log2f;
  * C with the GPU's exponents injected into the oracle: within 2 ulp (both
    sides run the same FP64 operation sequence, so 0 is expected);
  * |AB - C| within the Theorem 2 bound on every entry (plus half an ulp of
    the smallest subnormal where the output underflows, which the paper's
    analysis leaves out).
"""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import integer_matrix, paper_pair, wide_exponent_matrix

from _gpu_util import run_gpu, ulp_distance

pytestmark = pytest.mark.gpu

ULP_TOL = 2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2602_02549_b300.build import build
    build()


def check_against_oracle(oracle, A, Bm, g, b=64, bound=True):
    """Oracle with the GPU's mu, nu, N: W bit-exact, C within ULP_TOL, bound holds."""
    N = g["N"]
    r = oracle.os_ii(A, Bm, N, b, mu_in=g["mu"], nu_in=g["nu"])
    assert np.array_equal(g["W"], r["W"]), "W_l differs"
    d = ulp_distance(g["C"], r["C"], fp32=(b == 32))
    assert d.max() <= ULP_TOL, f"max ulp distance {d.max()}"
    assert oracle.lemma0_holds(r["Ap"], r["Bp"], N)
    if bound:
        eb = oracle.bound_from_exponents(A, Bm, g["mu"], g["nu"], r["Ap"], r["Bp"], N, b)
        eb = eb + (2.0 ** -1075 if b == 64 else 2.0 ** -150)
        err = np.abs(oracle.exact_residual(A, Bm, g["C"]))
        assert (err <= eb).all(), f"bound violated: max ratio {(err / eb).max()}"
    return r


SHAPES = [(1, 1, 1), (1, 7, 5), (9, 1, 3), (33, 65, 17), (128, 256, 64), (129, 257, 65),
          (200, 300, 1500), (256, 256, 256), (130, 40, 2049)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("N", [2, 14])
def test_dgemm_parity(oracle, shape, N):
    m, n, k = shape
    A, Bm = paper_pair(m, n, k, 0.5, seed=m + n + k)
    g = run_gpu(A, Bm, N)
    assert g["N"] == N
    r = check_against_oracle(oracle, A, Bm, g)
    # the exponents satisfy Algorithm 2 within the log2f band
    lo, hi = oracle.mu_band(r["mu_p"], r["cmax_row"], N)
    assert ((g["mu"] >= lo) & (g["mu"] <= hi)).all()
    lo, hi = oracle.mu_band(r["nu_p"], r["cmax_col"], N)
    assert ((g["nu"] >= lo) & (g["nu"] <= hi)).all()


@pytest.mark.parametrize("shape,N", [((4200, 300, 200), 5), ((8300, 70, 130), 14), ((16390, 33, 40), 17)])
def test_tall_problems(oracle, shape, N):
    # many row tiles (up to 129) and ragged last tiles in both directions
    m, n, k = shape
    A, Bm = paper_pair(m, n, k, 1.0, seed=m)
    g = run_gpu(A, Bm, N)
    check_against_oracle(oracle, A, Bm, g, bound=(m * n * k < 2e8))


# the bit length of |A'| grows with N: N <= 14 stays below 2^65 here, N = 20
# near 2^75, N = 24..28 between 2^78 and 2^104, N >= 33 above (every residue
# path of the kernels)
@pytest.mark.parametrize("N", [3, 5, 6, 8, 20, 24, 26, 28, 33, 49])
def test_dgemm_parity_moduli(oracle, N):
    A, Bm = paper_pair(150, 170, 700, 1.0, seed=N)
    g = run_gpu(A, Bm, N)
    check_against_oracle(oracle, A, Bm, g)


@pytest.mark.parametrize("phi", [0.5, 1.0, 2.0, 4.0])
def test_dgemm_phi(oracle, phi):
    A, Bm = paper_pair(96, 80, 1100, phi, seed=int(phi * 8))
    g = run_gpu(A, Bm, 16)
    check_against_oracle(oracle, A, Bm, g)


def test_exponents_match_oracle_log2f(oracle):
    # GPU __log2f vs the C library's log2f: mu, nu agree except in rows where
    # the two round across an integer boundary (counted; at most 2 allowed)
    A, Bm = paper_pair(256, 256, 512, 1.0, seed=5)
    g = run_gpu(A, Bm, 14)
    s = oracle.scaling(A, Bm, 14)
    mism = int((g["mu"] != s["own_mu"]).sum() + (g["nu"] != s["own_nu"]).sum())
    assert mism <= 2


@pytest.mark.parametrize("tr", [(True, False), (False, True), (True, True)])
def test_transposes(tr):
    ta, tb = tr
    A, Bm = paper_pair(70, 90, 300, 1.0, seed=3)
    As = np.ascontiguousarray(A.T) if ta else A
    Bs = np.ascontiguousarray(Bm.T) if tb else Bm
    g = run_gpu(As, Bs, 14, trans_a=ta, trans_b=tb)
    ref = run_gpu(A, Bm, 14)
    assert np.array_equal(g["C"], ref["C"])
    assert np.array_equal(g["mu"], ref["mu"]) and np.array_equal(g["nu"], ref["nu"])


@pytest.mark.parametrize("N", [2, 8, 14, 20, 33, 49])
def test_sgemm_parity(oracle, N):
    A, Bm = paper_pair(100, 140, 900, 1.0, seed=N, dtype=np.float32)
    g = run_gpu(A, Bm, N, fp32=True)
    check_against_oracle(oracle, A.astype(np.float64), Bm.astype(np.float64), g, b=32)


def test_integer_inputs_exact():
    # A' = 2^mu A exactly when mu >= 0; for N <= 5 every step is exact
    A = integer_matrix(90, 70, -30, 30, seed=1)
    Bm = integer_matrix(70, 110, -30, 30, seed=2)
    g = run_gpu(A, Bm, 5)
    assert (g["mu"] >= 0).all() and (g["nu"] >= 0).all()
    assert np.array_equal(g["C"], A @ Bm)


def test_extreme_residues_long_k(oracle):
    # injected mu = nu = 0 keeps A' = A; entries 127 / -128 drive every residue
    # to (near) its extreme, and k = 2^17 makes C'_1 = 2^31 (wraps in INT32 for
    # p = 256, still exact mod 256); closed form: every entry is k*a*b.
    k = 1 << 17
    for a, b in ((127.0, 127.0), (-128.0, -128.0), (127.0, -128.0)):
        A = np.full((4, k), a)
        Bm = np.full((k, 3), b)
        N = 8
        g = run_gpu(A, Bm, N, mu_in=np.zeros(4, np.int32), nu_in=np.zeros(3, np.int32))
        assert (g["C"] == k * a * b).all()
        r = oracle.os_ii(A, Bm, N, mu_in=np.zeros(4, np.int32), nu_in=np.zeros(3, np.int32))
        assert np.array_equal(g["W"], r["W"])


def test_random_integer_residue_products(oracle):
    # injected mu = nu = 0: A' = A, so W_l checks the tensor-core products alone
    A = integer_matrix(130, 3000, -(1 << 40), 1 << 40, seed=7)
    Bm = integer_matrix(3000, 260, -(1 << 40), 1 << 40, seed=8)
    g = run_gpu(A, Bm, 12, mu_in=np.zeros(130, np.int32), nu_in=np.zeros(260, np.int32))
    r = oracle.os_ii(A, Bm, 12, mu_in=np.zeros(130, np.int32), nu_in=np.zeros(260, np.int32))
    assert np.array_equal(g["W"], r["W"])
    assert ulp_distance(g["C"], r["C"]).max() <= ULP_TOL


@pytest.mark.parametrize("N,b,bits", [(2, 64, 20), (3, 64, 20), (5, 64, 20), (9, 64, 45), (12, 64, 50),
                                       (2, 32, 20), (3, 32, 20), (5, 32, 20)])
def test_q_near_half_integers(oracle, N, b, bits):
    # injected mu = nu = 0 with |A'B'| far above P/2: C' wraps mod P, so
    # P_inv C'(1) spreads evenly over whole intervals and about one entry in 128
    # lies within 2^-8 of a half-integer, where the rounding of the FP64 product
    # and the round-half-even of Q (taken on the integer units) decide Q.  Every
    # entry must still equal the oracle's (0 ulp: both take the same FP64 steps).
    m, n, k = 96, 160, 300
    A = integer_matrix(m, k, -(1 << bits), 1 << bits, seed=N)
    Bm = integer_matrix(k, n, -(1 << bits), 1 << bits, seed=N + 100)
    zm, zn = np.zeros(m, np.int32), np.zeros(n, np.int32)
    g = run_gpu(A, Bm, N, fp32=(b == 32), mu_in=zm, nu_in=zn)
    r = oracle.os_ii(A, Bm, N, b, mu_in=zm, nu_in=zn)
    assert np.array_equal(g["W"], r["W"])
    assert ulp_distance(g["C"], r["C"], fp32=(b == 32)).max() == 0
    y = oracle.constants(N, b).Pinv * r["C1"]
    near = np.abs(np.abs(y - np.rint(y)) - 0.5) < 2.0 ** -8
    assert near.sum() >= 20, "the inputs no longer come near half-integers"


def test_wide_exponents_and_zeros(oracle):
    A = wide_exponent_matrix(70, 300, -1060, 400, seed=9, zero_frac=0.3)
    Bm = wide_exponent_matrix(300, 50, -900, 400, seed=10, zero_frac=0.3)
    A[5, :] = 0.0
    Bm[:, 7] = 0.0
    g = run_gpu(A, Bm, 20)
    check_against_oracle(oracle, A, Bm, g)
    assert (g["C"][5] == 0).all() and (g["C"][:, 7] == 0).all()


def test_subnormal_rows(oracle):
    # rows made only of subnormal numbers (mu near 1074 + 60: the residue
    # kernels shift significands without the implicit bit into x' of at most
    # 64 bits), rows mixing subnormals with normal values, the smallest
    # subnormals, a zero row and a subnormal column of B, at N where every
    # row stays below 2^64; then the transposed layouts give the same bits
    A, Bm = paper_pair(37, 29, 150, 1.0, seed=21)
    A[3, :] = np.ldexp(A[3, :], -1040)
    A[7, ::2] = np.ldexp(A[7, ::2], -1060)
    A[11, :] = 0.0
    A[13, :40] = 5e-324 * np.arange(1, 41)
    A[13, 40:] = 0.0
    Bm[:, 4] = np.ldexp(Bm[:, 4], -1050)
    assert (np.abs(A[3]) < 2.0 ** -1022).all() and (A[3] != 0).any()
    for N in (14, 16):
        g = run_gpu(A, Bm, N)
        check_against_oracle(oracle, A, Bm, g)
        gt = run_gpu(np.ascontiguousarray(A.T), np.ascontiguousarray(Bm.T), N, trans_a=True, trans_b=True)
        assert np.array_equal(gt["C"], g["C"]) and np.array_equal(gt["W"], g["W"])


def test_zero_operands(oracle):
    # A = 0, B = 0 or both: every row uses Dbar = 1 (reading of Algorithm 2 for
    # a zero Cbar row), every bound term and L vanish, so the rule takes N = 2
    # as the oracle's does, W is zero and C exactly zero, in every mode
    A, Bm = paper_pair(20, 30, 40, 1.0, seed=3)
    Z, Zb = np.zeros_like(A), np.zeros_like(Bm)
    for X, Y in ((Z, Bm), (A, Zb), (Z, Zb)):
        s = oracle.scaling(X, Y, 14)
        N_or, _ = oracle.choose_N(X, Y, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], 1e-15, 20)
        for N, fast in ((14, False), (0, False), (0, True)):
            g = run_gpu(X, Y, N, target=1e-15, nmax=20, fast=fast)
            if N == 0 and not fast:
                assert g["N"] == N_or == 2
            assert (g["C"] == 0).all() and not np.isnan(g["C"]).any()
            assert (g["W"] == 0).all()
            check_against_oracle(oracle, X, Y, g)


def test_non_finite_inputs_complete():
    # NaN or Inf inputs break the paper's preconditions and their results are
    # unspecified; the call must still complete (OZ2_OK, a clean sync) and
    # leave the library working: the same finite call gives the same bits
    # before and after
    import torch
    from paper_2602_02549_b300 import binding as B
    A, Bm = paper_pair(70, 50, 300, 1.0, seed=31)
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(Bm, device="cuda")
    C0 = B.matmul(At, Bt, 14)
    torch.cuda.synchronize()
    bad_A, bad_B = At.clone(), Bt.clone()
    bad_A[3, :] = float("inf")
    bad_A[9, 17] = float("nan")
    bad_B[:, 5] = -float("inf")
    bad_B[100, 20] = float("nan")
    for X, Y in ((bad_A, Bt), (At, bad_B), (bad_A, bad_B)):
        for N, mode in ((14, 0), (0, 0), (0, B.OZ2_FAST)):
            C = torch.empty((70, 50), dtype=torch.float64, device="cuda")
            assert B.gemm_ex(X, Y, C, N, mode, target=1e-15 if N == 0 else 0.0, nmax=20 if N == 0 else 0) == 0
            torch.cuda.synchronize()
            assert B.sync() == 0
    C1 = B.matmul(At, Bt, 14)
    torch.cuda.synchronize()
    assert torch.equal(C0, C1)


def test_subnormal_outputs(oracle):
    # tiny inputs make C subnormal: the single final rounding must match ldexp
    A, Bm = paper_pair(40, 30, 200, 1.0, seed=4)
    A = np.ldexp(A, -530)
    Bm = np.ldexp(Bm, -530)
    g = run_gpu(A, Bm, 14)
    assert (np.abs(g["C"]) < 2.0 ** -1022).mean() > 0.5
    check_against_oracle(oracle, A, Bm, g)


def test_auto_N_rule(oracle):
    for phi, tau in ((0.5, 1e-15), (1.0, 1e-15), (2.0, 1e-12), (1.0, 1e-8)):
        A, Bm = paper_pair(128, 128, 1024, phi, seed=int(phi * 3))
        g = run_gpu(A, Bm, 0, target=tau, nmax=40)
        s = oracle.scaling(A, Bm, 14)
        N, info = oracle.choose_N(A, Bm, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], tau, 40)
        rat = info["ratios"]
        slack = 1e-9
        assert rat[g["N"]] <= tau * (1 + slack) or g["N"] == 40
        if g["N"] > 2:
            assert rat[g["N"] - 1] > tau * (1 - slack)
        check_against_oracle(oracle, A, Bm, g)


@pytest.mark.parametrize("phi,tau", [(1.0, 1e-7), (0.5, 1e-6), (2.0, 1e-5), (1.0, 1e-3)])
def test_auto_N_rule_sgemm(oracle, phi, tau):
    A, Bm = paper_pair(128, 160, 1024, phi, seed=int(phi * 7), dtype=np.float32)
    g = run_gpu(A, Bm, 0, fp32=True, target=tau, nmax=20)
    A, Bm = A.astype(np.float64), Bm.astype(np.float64)
    s = oracle.scaling(A, Bm, 14, 32)
    N, info = oracle.choose_N(A, Bm, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], tau, 20, 32)
    rat = info["ratios"]
    assert rat[g["N"]] <= tau * (1 + 1e-9) or g["N"] == 20, (g["N"], N, rat)
    if g["N"] > 2:
        assert rat[g["N"] - 1] > tau * (1 - 1e-9), (g["N"], N, rat)
    check_against_oracle(oracle, A, Bm, g, b=32)


def test_deterministic():
    A, Bm = paper_pair(300, 200, 800, 1.0, seed=1)
    a = run_gpu(A, Bm, 0, target=1e-15)
    b = run_gpu(A, Bm, 0, target=1e-15)
    assert a["N"] == b["N"]
    assert np.array_equal(a["C"].view(np.int64), b["C"].view(np.int64))


def test_log2f_assumption():
    # Section 1.2, assumption (1), for the __log2f the exponent kernel uses
    from paper_2602_02549_b300 import binding as B
    viol, ratio = B.check_log2f()
    assert viol == 0, f"{viol} violations, max |err|/(u32 log2 x) = {ratio}"
    assert ratio <= 4.0


@pytest.mark.parametrize("b", [64, 32])
@pytest.mark.parametrize("phi,N", [(0.5, 8), (1.0, 14), (2.0, 17), (4.0, 20)])
def test_fast_mode(oracle, phi, N, b):
    # fast mode: Cbar replaced by its Cauchy-Schwarz majorant (no scaling GEMM)
    dt = np.float64 if b == 64 else np.float32
    A, Bm = paper_pair(150, 210, 900, phi, seed=int(phi * 5) + N, dtype=dt)
    A, Bm = A.astype(np.float64), Bm.astype(np.float64)
    g = run_gpu(A.astype(dt), Bm.astype(dt), N, fp32=(b == 32), fast=True)
    check_against_oracle(oracle, A, Bm, g, b=b)
    s = oracle.scaling(A, Bm, N, b, fast=True)
    lo, hi = oracle.mu_band(s["mu_p"], s["cmax_row"], N, b)
    assert ((g["mu"] >= lo) & (g["mu"] <= hi)).all()
    lo, hi = oracle.mu_band(s["nu_p"], s["cmax_col"], N, b)
    assert ((g["nu"] >= lo) & (g["nu"] <= hi)).all()


def test_fast_mode_auto_N(oracle):
    A, Bm = paper_pair(128, 160, 700, 1.0, seed=9)
    g = run_gpu(A, Bm, 0, target=1e-14, nmax=30, fast=True)
    s = oracle.scaling(A, Bm, 14, fast=True)
    _, info = oracle.choose_N(A, Bm, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], 1e-14, 30)
    assert info["ratios"][g["N"]] <= 1e-14 * (1 + 1e-9)
    assert info["ratios"][g["N"] - 1] > 1e-14 * (1 - 1e-9)
    check_against_oracle(oracle, A, Bm, g)


@pytest.mark.parametrize("b,N", [(64, 8), (64, 17), (64, 20), (32, 9), (32, 14)])
def test_vs_fma_chain_reading(oracle, b, N):
    # the other reading of fl(sum) in Algorithm 3 (fma chains in ascending l).
    # DGEMM: C'(1) is exact in both and C'(2) only feeds the last bits, so the
    # results stay within ULP_TOL.  SGEMM: C'(1) itself differs by up to about
    # N u_64 rho P (the first term of R_32, Lemma 4), which is many FP32 ulp on
    # entries far below their row and column maxima; both results must then
    # satisfy Theorem 2's bound.
    dt = np.float64 if b == 64 else np.float32
    A, Bm = paper_pair(200, 300, 1500, 1.0, seed=N + 100, dtype=dt)
    g = run_gpu(A, Bm, N, fp32=(b == 32))
    A, Bm = A.astype(np.float64), Bm.astype(np.float64)
    r = oracle.os_ii(A, Bm, N, b, mu_in=g["mu"], nu_in=g["nu"], fma_chain=True)
    assert np.array_equal(g["W"], r["W"])
    if b == 64:
        assert ulp_distance(g["C"], r["C"]).max() <= ULP_TOL
    else:
        eb = oracle.bound_from_exponents(A, Bm, g["mu"], g["nu"], r["Ap"], r["Bp"], N, b) + 2.0 ** -150
        for C in (g["C"], np.asarray(r["C"], np.float64)):
            assert (np.abs(oracle.exact_residual(A, Bm, C)) <= eb).all()


@pytest.mark.parametrize("N,phi", [(16, 1.0), (17, 0.5), (17, 1.0), (17, 4.0), (18, 4.0), (20, 4.0),
                                   (21, 1.0), (27, 1.0), (28, 0.5), (28, 1.0), (33, 1.0)])
def test_short_rows_limb_thresholds(oracle, N, phi):
    # k = 20 (k_pad = 64): one warp of the residue kernels covers four rows.
    # Across these N the bit length of the rows' largest |A'|, |B'| passes the
    # 64 / 65 / 78 / 104 bit limits of the 64-bit and 128-bit 5-limb forms and
    # the 6- and 8-limb forms (N = 16: 61 to 62 bits); at N = 17, phi = 0.5 (64
    # or 65 bits), N = 17, phi = 1 (65 or 66) and N = 28, phi = 0.5 (104 to 106)
    # neighbouring rows lie on both sides of a limit.  W must stay bit-exact
    A, Bm = paper_pair(130, 70, 20, phi, seed=N)
    g = run_gpu(A, Bm, N)
    check_against_oracle(oracle, A, Bm, g)
    As, Bs = np.ascontiguousarray(A.T), np.ascontiguousarray(Bm.T)
    gt = run_gpu(As, Bs, N, trans_a=True, trans_b=True)
    assert np.array_equal(gt["C"], g["C"]) and np.array_equal(gt["W"], g["W"])


@pytest.mark.parametrize("phi", [0.5, 1.0, 2.0, 4.0])
def test_paper_shape_error_vs_bounds(oracle, phi):
    # the paper's shape for its error-versus-bound comparison (m = n = 128,
    # k = 8192): per N, the measured error of the GPU's C against the exact
    # product, divided by the bound of eq. thm:err-1 and eq. thm:err-2 (the
    # oracle's own scaling) and by the Lemma 1 + Lemma 4 bound from the GPU's
    # exponents; the mu / nu mismatch count against the oracle's own exponents
    A, Bm = paper_pair(128, 128, 8192, phi, seed=int(phi * 10))
    for N in (8, 14, 20):
        g = run_gpu(A, Bm, N)
        check_against_oracle(oracle, A, Bm, g)
        own = oracle.os_ii(A, Bm, N)
        mism = int((g["mu"] != own["mu"]).sum() + (g["nu"] != own["nu"]).sum())
        assert mism <= 2
        err = np.abs(oracle.exact_residual(A, Bm, g["C"]))
        e1, e2 = oracle.bounds(A, Bm, own)
        eb = oracle.bound_from_exponents(A, Bm, g["mu"], g["nu"], own["Ap"], own["Bp"], N) \
            if mism == 0 else None
        r1, r2 = float((err / e1).max()), float((err / e2).max())
        if mism == 0:
            assert r1 <= 1.0 and r2 <= 1.0
        print(f"phi={phi} N={N} mu/nu mismatches={mism} max err/err1={r1:.3e} max err/err2={r2:.3e}"
              + (f" max err/bound(exponents)={float((err / eb).max()):.3e}" if eb is not None else ""))
