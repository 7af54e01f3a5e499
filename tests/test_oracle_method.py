"""Pins of the CPU oracle (Algorithms 1-3) against exact mathematics.

* exact rationals (Python Fraction / int) on tiny inputs: the exact product,
  A'B' both directly and through the CRT, Lemmas 0-4 and Theorem 2;
* integer-valued inputs that must come out exact (N <= 5, where s_l2 = P2 = 0);
* the superaccumulator against Fraction sums;
* planted mistakes (in the oracle's tables, on the CPU) that these pins catch.
"""
import dataclasses
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle.constants import U32, U64, bound_terms, constants
from paper_2602_02549_b300.inputs import (integer_matrix, paper_pair, paper_matrix,
                                          wide_exponent_matrix)


def frac_matmul(A, B):
    m, k = A.shape
    n = B.shape[1]
    FA = [[Fraction(float(A[i, h])) for h in range(k)] for i in range(m)]
    FB = [[Fraction(float(B[h, j])) for j in range(n)] for h in range(k)]
    return [[sum(FA[i][h] * FB[h][j] for h in range(k)) for j in range(n)] for i in range(m)]


def int_matmul(Ap, Bp):
    m, k = Ap.shape
    n = Bp.shape[1]
    IA = [[int(Ap[i, h]) for h in range(k)] for i in range(m)]
    IB = [[int(Bp[h, j]) for j in range(n)] for h in range(k)]
    return ([[sum(IA[i][h] * IB[h][j] for h in range(k)) for j in range(n)] for i in range(m)],
            [[sum(abs(IA[i][h] * IB[h][j]) for h in range(k)) for j in range(n)] for i in range(m)])


def t_frac_up(P):
    # t = 1/sqrt(32 (P-1)), as a rational upper bound
    t = Fraction(1.0 / math.sqrt(32.0 * float(P - 1))) * (1 + Fraction(1, 1 << 45))
    assert t * t * 32 * (P - 1) >= 1
    return t


# --------------------------------------------------------------------------- #
def test_exact_residual_matches_fractions(oracle):
    rng = np.random.default_rng(7)
    for trial in range(30):
        k = int(rng.integers(1, 40))
        x = wide_exponent_matrix(1, k, -1074, 520, seed=trial)
        y = wide_exponent_matrix(k, 1, -600, 490, seed=100 + trial)
        if trial % 3 == 0:                       # heavy cancellation
            y[:, 0] = 1.0
            x[0, k // 2:] = -x[0, :k - k // 2]
        if trial % 5 == 0:                       # subnormal-only
            x = np.ldexp(np.round(rng.random((1, k)) * 1000), -1074)
            y = np.ones((k, 1))
        c = float(rng.standard_normal()) * 2.0 ** int(rng.integers(-1000, 1000))
        c = c if abs(c) < 1e300 else 1.0
        exact = sum(Fraction(float(x[0, h])) * Fraction(float(y[h, 0])) for h in range(k))
        got = oracle.exact_residual(x, y)[0, 0]
        assert got == float(exact)
        got_c = oracle.exact_residual(x, y, np.array([[c]]))[0, 0]
        assert got_c == float(exact - Fraction(c))


def test_exact_abs_sums(oracle):
    X = wide_exponent_matrix(5, 33, -1070, 900, seed=3)
    got = oracle.abs_sums(X, axis=1)
    for i in range(5):
        assert got[i] == float(sum(abs(Fraction(float(v))) for v in X[i]))


def test_residues_match_python_ints(oracle):
    rng = np.random.default_rng(1)
    vals = []
    for e in list(range(0, 180, 3)):
        for _ in range(4):
            vals.append(float(np.ldexp(rng.random() + 1.0, e)))
    vals = np.trunc(np.array(vals + [0.0, 1.0, 127.0, 128.0, 255.0, 256.0, 2.0 ** 53 - 1]))
    vals = np.concatenate([vals, -vals])
    for p in constants(49).p:
        got = oracle.residues(vals, p)
        for v, g in zip(vals, got):
            r = int(v) % p
            if 2 * r > p:
                r -= p
            if p == 256 and r == 128:
                r = -128
            assert g == r
            assert -(p // 2) <= g <= p // 2


def test_exponent_shift_exact(oracle):
    rng = np.random.default_rng(2)
    for N in (2, 14, 49):
        C = constants(N)
        e = (rng.random(2000) * 31).astype(np.float32)
        got = oracle.exponent_shift(C.c, e, C.Pprime)
        for ei, g in zip(e, got):
            v = Fraction(float(C.c)) * Fraction(float(ei)) + Fraction(float(C.Pprime))
            assert g == math.floor(v)


# --------------------------------------------------------------------------- #
CASES = [(3, 4, 5, 0.5), (5, 3, 7, 1.0), (4, 4, 6, 2.0), (2, 6, 3, 4.0), (6, 5, 1, 1.0)]


@pytest.mark.parametrize("b", [64, 32])
@pytest.mark.parametrize("N", [2, 3, 5, 8, 14, 20, 49])
@pytest.mark.parametrize("case", CASES)
def test_tiny_bruteforce(oracle, case, N, b):
    m, n, k, phi = case
    dt = np.float64 if b == 64 else np.float32
    A, B = paper_pair(m, n, k, phi, seed=N * 7 + m, dtype=dt)
    A, B = A.astype(np.float64), B.astype(np.float64)
    r = oracle.os_ii(A, B, N, b)
    C = constants(N, b)
    P = C.P
    # exact A'B' directly, and via the CRT of the W_l (Theorem 1, Lemma 3 proof)
    ApBp, absApBp = int_matmul(r["Ap"], r["Bp"])
    crtAB, Qx = oracle.crt_exact(r["W"], N)
    t = t_frac_up(P)
    AB = frac_matmul(A, B)
    rho = C.rho
    for i in range(m):
        for j in range(n):
            e = i * n + j
            # Lemma 0: |A'||B'| < P/2
            assert 2 * absApBp[i][j] < P
            assert crtAB[e] == ApBp[i][j]
            # Lemma 3: Q == round(sum q_l/p_l W_l)
            assert r["Q"][i, j] == Qx[e]
            W = [int(r["W"][l, i, j]) for l in range(N)]
            Sx = sum(xl * w for xl, w in zip(C.x, W))
            if b == 64:
                # Lemma 2: C'(1) exact, and the bound on C'(1) + C'(2)
                assert Fraction(r["C1"][i, j]) == sum(Fraction(s) * w for s, w in zip(C.s1, W))
                lhs = abs(Fraction(r["C1"][i, j]) + Fraction(r["C2"][i, j]) - Sx)
                assert lhs <= Fraction(2) ** (1 + (rho - 1).bit_length()) * (N + 1 + N * U64) * U64 ** 2 * rho * P
                Rb = (1 + 3 * U64) * Fraction(2) ** (1 + (rho - 1).bit_length()) * (N + 2) * U64 ** 2 * rho * P \
                    + 3 * U64 * abs(ApBp[i][j])
            else:
                assert abs(Fraction(r["C1"][i, j]) - Sx) <= (N + 1) * U64 * rho * P
                Rb = (1 + U32) * (N + 2) * U64 * rho * P + U32 * abs(ApBp[i][j])
            # Lemma 4: |A'B' - C''| <= R_b
            assert abs(ApBp[i][j] - Fraction(r["Cpp"][i, j])) <= Rb
            # Theorem 2, eq. thm:err-1
            if r["alpha"][i] == oracle.INT32_MIN or r["beta"][j] == oracle.INT32_MIN:
                continue
            ep = Fraction(int(r["cmax_row"][i]))
            fp = Fraction(int(r["cmax_col"][j]))
            # 2^alpha' = 2^alpha sqrt(max cbar); use exact upper bounds of the square roots
            sa = Fraction(math.isqrt(int(ep)) + 1)
            sb = Fraction(math.isqrt(int(fp)) + 1)
            a2 = Fraction(2) ** int(r["alpha"][i]) * sa
            b2 = Fraction(2) ** int(r["beta"][j]) * sb
            Ra = sum(abs(Fraction(float(v))) for v in A[i])
            Kb = sum(abs(Fraction(float(v))) for v in B[:, j])
            err1 = t * Ra * b2 + t * a2 * Kb + (k + Rb) * t * t * a2 * b2
            Cij = Fraction(float(r["C"][i, j]))
            assert abs(AB[i][j] - Cij) <= err1
    # Lemma 1: mu_i >= -alpha'_i + (log2(P-1) + 5)/2
    assert oracle.ozaki_exponent_floor_ok(r["mu"], r["alpha"], r["cmax_row"], N).all()
    assert oracle.ozaki_exponent_floor_ok(r["nu"], r["beta"], r["cmax_col"], N).all()


@pytest.mark.parametrize("N", [2, 3, 4, 5])
@pytest.mark.parametrize("shape", [(7, 5, 4), (16, 9, 8), (3, 11, 2), (1, 1, 1)])
def test_integer_inputs_exact(oracle, N, shape):
    # A' = 2^mu A exactly when mu >= 0; for N <= 5, s_l2 = P2 = 0 and every step
    # of Algorithm 3 is exact, so C must equal AB bit for bit.
    m, n, k = shape
    A = integer_matrix(m, k, -30, 30, seed=m + N)
    B = integer_matrix(k, n, -30, 30, seed=n + 10 * N)
    r = oracle.os_ii(A, B, N, 64)
    assert (r["mu"] >= 0).all() and (r["nu"] >= 0).all()
    assert np.array_equal(r["C"], A @ B)


@pytest.mark.parametrize("b", [64, 32])
@pytest.mark.parametrize("N", [2, 6, 14, 20])
@pytest.mark.parametrize("phi", [0.5, 1.0, 2.0, 4.0])
def test_bound_holds(oracle, phi, N, b):
    # Theorem 2 on every entry, eq. thm:err-1 <= eq. thm:err-2
    dt = np.float64 if b == 64 else np.float32
    A, B = paper_pair(24, 20, 300, phi, seed=int(phi * 10) + N, dtype=dt)
    r = oracle.os_ii(A, B, N, b)
    err = np.abs(oracle.exact_residual(A.astype(np.float64), B.astype(np.float64), r["C"]))
    e1, e2 = oracle.bounds(A.astype(np.float64), B.astype(np.float64), r)
    assert (err <= e1).all()
    assert (e1 <= e2 * (1 + 1e-12)).all()


def test_bound_holds_wide_exponents(oracle):
    A = wide_exponent_matrix(12, 40, -1000, 450, seed=5, zero_frac=0.2)
    B = wide_exponent_matrix(40, 10, -900, 450, seed=6, zero_frac=0.2)
    for N in (3, 14, 49):
        r = oracle.os_ii(A, B, N, 64)
        err = np.abs(oracle.exact_residual(A, B, r["C"]))
        e1, _ = oracle.bounds(A, B, r)
        assert (err <= e1).all()


def test_degenerate_rows_and_columns(oracle):
    A, B = paper_pair(6, 5, 8, 1.0, seed=3)
    A[2, :] = 0.0                  # zero row of A
    B[:, 4] = 0.0                  # zero column of B
    B[1, :] = 0.0                  # row of B that row 0 of A alone hits
    A[0, :] = 0.0
    A[0, 1] = 3.0
    r = oracle.os_ii(A, B, 14, 64)
    assert (r["C"][2] == 0).all() and (r["C"][:, 4] == 0).all() and (r["C"][0] == 0).all()
    err = np.abs(oracle.exact_residual(A, B, r["C"]))
    e1, _ = oracle.bounds(A, B, r)
    assert (err <= e1).all()


def test_own_mu_within_band(oracle):
    A, B = paper_pair(40, 30, 500, 1.0, seed=11)
    for N in (2, 14, 49):
        r = oracle.os_ii(A, B, N)
        lo, hi = oracle.mu_band(r["mu_p"], r["cmax_row"], N)
        assert ((r["mu"] >= lo) & (r["mu"] <= hi)).all()
        lo, hi = oracle.mu_band(r["nu_p"], r["cmax_col"], N)
        assert ((r["nu"] >= lo) & (r["nu"] <= hi)).all()


def test_choose_N_self_consistent(oracle):
    for phi in (0.5, 1.0, 2.0):
        A, B = paper_pair(32, 32, 512, phi, seed=int(phi * 4))
        s = oracle.scaling(A, B, 14)
        for tau in (1e-8, 1e-12, 1e-15):
            N, info = oracle.choose_N(A, B, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], tau, 49)
            assert info["ratios"][N] <= tau or N == 49
            if N > 2:
                assert info["ratios"][N - 1] > tau
            # the normwise error at that N stays within the target plus the N-independent floor
            r = oracle.os_ii(A, B, N)
            err = np.abs(oracle.exact_residual(A, B, r["C"])).max()
            absAB = oracle.exact_product(np.abs(A), np.abs(B)).max()
            floor = bound_terms(N)["rb"] * bound_terms(N)["t"] ** 2 * info["max2a"] * info["max2b"]
            assert err <= tau * absAB + floor


# --------------------------------------------------------------------------- #
# Planted mistakes: each must be caught by one of the pins above.
# --------------------------------------------------------------------------- #
def test_planted_mistakes_are_caught(oracle):
    A, B = paper_pair(8, 8, 64, 1.0, seed=21)
    N = 14
    good = constants(N)
    ref = oracle.os_ii(A, B, N)
    ApBp, _ = int_matmul(ref["Ap"], ref["Bp"])

    def lemma4_ok(r, C):
        rho = C.rho
        for i in range(8):
            for j in range(8):
                Rb = (1 + 3 * U64) * Fraction(2) ** (1 + (rho - 1).bit_length()) * (N + 2) * U64 ** 2 * rho * C.P \
                    + 3 * U64 * abs(ApBp[i][j])
                if abs(ApBp[i][j] - Fraction(r["Cpp"][i, j])) > Rb:
                    return False
        return True

    assert lemma4_ok(ref, good)
    # (a) dropped low part C'(2)
    bad = dataclasses.replace(good, s2=tuple(0.0 for _ in good.s2))
    assert not lemma4_ok(oracle.crt_from_W(ref["W"], N, consts=bad), good)
    # (b) wrong sign of P2
    bad = dataclasses.replace(good, P2=-good.P2)
    assert not lemma4_ok(oracle.crt_from_W(ref["W"], N, consts=bad), good)
    # (c) wrong inverse q_1: the CRT round trip fails
    badx = list(good.x)
    badx[1] = (good.P // good.p[1]) * ((good.q[1] + 1) % good.p[1])
    x = 12345678901234
    ys = [x % pl for pl in good.p]
    S = sum(xl * y for xl, y in zip(badx, ys)) % good.P
    assert S != x
    # (d) transposed operand: the Theorem 2 bound fails
    As, Bs = paper_pair(16, 16, 16, 1.0, seed=22)
    refs = oracle.os_ii(As, Bs, N)
    r = oracle.os_ii(As, Bs.T.copy(), N)
    err = np.abs(oracle.exact_residual(As, Bs, r["C"]))
    e1, _ = oracle.bounds(As, Bs, refs)
    assert not (err <= e1).all()
    # (e) exponents one too large: Lemma 0 (|A'||B'| < P/2) fails somewhere
    s = oracle.scaling(A, B, N)
    r = oracle.os_ii(A, B, N, mu_in=s["mu"] + 2, nu_in=s["nu"] + 2)
    _, absApBp = int_matmul(r["Ap"], r["Bp"])
    assert max(max(row) for row in absApBp) * 2 >= good.P


# --------------------------------------------------------------------------- #
# Fast mode (a reading: Cbar replaced by its Cauchy-Schwarz majorant)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("b", [64, 32])
@pytest.mark.parametrize("N", [2, 6, 14, 20, 49])
@pytest.mark.parametrize("phi", [0.5, 2.0, 4.0])
def test_fast_mode_bound_and_lemma0(oracle, phi, N, b):
    dt = np.float64 if b == 64 else np.float32
    A, B = paper_pair(20, 24, 260, phi, seed=int(phi * 7) + N, dtype=dt)
    A, B = A.astype(np.float64), B.astype(np.float64)
    r = oracle.os_ii(A, B, N, b, fast=True)
    exact = oracle.scaling(A, B, N, b)
    # the majorant dominates Cbar (Cauchy-Schwarz) and stays <= 2^12 k
    assert (r["cmax_row"] >= exact["cmax_row"]).all() and (r["cmax_col"] >= exact["cmax_col"]).all()
    assert r["cmax_row"].max() <= 4096 * A.shape[1]
    assert oracle.lemma0_holds(r["Ap"], r["Bp"], N)
    assert oracle.ozaki_exponent_floor_ok(r["mu"], r["alpha"], r["cmax_row"], N).all()
    err = np.abs(oracle.exact_residual(A, B, r["C"]))
    e1, _ = oracle.bounds(A, B, r)
    assert (err <= e1).all()


def test_fast_mode_sum_of_squares_by_hand(oracle):
    # Abar rows (1, 2, 2) and (3, 0, 4): ||.||^2 = 9 and 25; Bbar columns
    # (2, 2, 1) and (0, 4, 3): 9 and 25.  Row maxima ceil(sqrt(9*25)) = 15 and
    # ceil(sqrt(25*25)) = 25, column maxima ceil(sqrt(25*9)) = 15 and 25.
    Abar = np.array([[1, 2, 2], [3, 0, 4]], np.int8)
    Bbar = np.array([[2, 0], [2, 4], [1, 3]], np.int8)
    row, col = oracle.fast_cbar_maxima(Abar, Bbar)
    assert list(row) == [15, 25] and list(col) == [15, 25]
    assert oracle.ceil_sqrt(10) == 4 and oracle.ceil_sqrt(16) == 4 and oracle.ceil_sqrt(0) == 0


@pytest.mark.parametrize("b", [64, 32])
@pytest.mark.parametrize("N", [2, 6, 9, 17, 33, 49])
def test_crt_sums_correctly_rounded(oracle, N, b):
    # Algorithm 3: C'(1) and C'(2) are the exact sums sum_l s_l W_l rounded once
    # to the nearest double; Python's int / int division is correctly rounded,
    # so the reference values below come from exact rational arithmetic alone.
    C = constants(N, b)
    rng = np.random.default_rng(N + b)
    lo = np.array([-(p // 2) for p in C.p])
    hi = np.array([(p - 1) // 2 for p in C.p])
    W = rng.integers(lo[:, None], hi[:, None] + 1, size=(N, 300)).astype(np.int8)
    W[:, 0] = lo.astype(np.int8)                  # all at the negative extreme
    W[:, 1] = hi.astype(np.int8)
    W[:, 2] = 0
    r = oracle.crt_from_W(W, N, b)

    def rounded(svals, col):
        num = sum(Fraction(s) * int(W[l, col]) for l, s in enumerate(svals))
        return num.numerator / num.denominator

    for e in range(W.shape[1]):
        assert r["C1"][e] == rounded(C.s1, e)
        assert r["C2"][e] == rounded(C.s2, e)
    assert r["C1"][2] == 0.0 and r["C2"][2] == 0.0


def test_crt_fma_chain_reading(oracle):
    # the other reading of fl(sum): an fma chain in ascending l.  It is checked
    # against fma steps emulated with exact rationals, and differs from the
    # correctly rounded C'(2) on some entries (so the test above pins which
    # reading the default takes), while C'' agrees to a few ulp.
    N, b = 17, 64
    C = constants(N, b)
    rng = np.random.default_rng(3)
    W = np.stack([rng.integers(-(p // 2), (p - 1) // 2 + 1, size=1500) for p in C.p]).astype(np.int8)
    r = oracle.crt_from_W(W, N, b)
    rc = oracle.crt_from_W(W, N, b, fma_chain=True)
    diff = 0
    for e in range(W.shape[1]):
        acc = 0.0
        for l in range(N):
            t = Fraction(C.s2[l]) * int(W[l, e]) + Fraction(acc)     # fma: one rounding
            acc = t.numerator / t.denominator
        assert rc["C2"][e] == acc
        diff += acc != r["C2"][e]
    assert diff > 0
    assert np.array_equal(rc["C1"], r["C1"])                  # exact either way (Lemma 2)
    d = np.abs(rc["Cpp"].view(np.int64) - r["Cpp"].view(np.int64))
    assert d.max() <= 2
