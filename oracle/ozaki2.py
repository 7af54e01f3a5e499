"""CPU oracle of the Ozaki-II scheme (arXiv 2602.02549), Algorithms 1-3.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the GPU library; the loops live in oracle/oz2_oracle.c (plain C) and the
constants in oracle/constants.py (Python integers).

The steps below follow the paper's order and notation:
  Algorithm 2 (Scaling):  mu', Abar, nu', Bbar, Cbar = Abar Bbar,
      Dbar = single_up(Cbar), e = log2f(max dbar), f likewise,
      mu = mu' + floor(fma_down(c, e, P')), A' = trunc(2^mu A), B' likewise.
  Algorithm 3 (CRT):  A'_l = mod(A', p_l), B'_l, C'_l = A'_l B'_l,
      W_l = mod(C'_l, p_l), C'(1), C'(2), Q, C''.
  Algorithm 1:  C = diag(2^-mu) C'' diag(2^-nu).

Readings where the paper is silent:
  * floor(fl_down(fma(c, e, P'))) equals floor(c*e + P') taken exactly, because
    rounding down never crosses the integer below; c*e + P' is exact in FP64.
  * A zero row of A (zero column of B) gets mu' = 0; a row whose Cbar row is
    all zero uses max dbar = 1 (e = 0).  The output there is exactly 0.
  * C'(1) and C'(2) are the exact sums rounded once (fma_chain=True: fma
    chains in ascending l from +0, the other reading of fl(sum)).
  * k > 2^17 (outside the paper's assumption, Section 3): split-K, one OS_II
    per range of consecutive k, results added in range order (os_ii_splitk).
  * The final scaling is one ldexp by -(mu_i + nu_j).  For b = 32 the
    rounding single(C'') of Algorithm 3 is applied after that scaling, which
    changes nothing unless single(C'') would overflow (P > 2^128, N >= 17) or
    C is subnormal.
  * e = log2f(.) is the C library's log2f unless exponents are injected.
"""
from __future__ import annotations

import ctypes
import math
from fractions import Fraction

import numpy as np

from . import build as _build
from .constants import MODULI, K_MAX, N_MAX, N_MIN, U32, bound_terms, constants

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        P = ctypes.c_void_p
        i32, i64, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
        _lib.oz2o_floor_log2_absmax.argtypes = [i32, i32, P, i64, i64, P]
        _lib.oz2o_ceil_scaled_abs.argtypes = [i32, i32, P, i64, i64, P, P]
        _lib.oz2o_gemm_i8_i64.argtypes = [i32, i32, i32, P, P, P]
        _lib.oz2o_trunc_scaled.argtypes = [i32, i32, P, i64, i64, P, P]
        _lib.oz2o_residues.argtypes = [i64, P, i32, P]
        _lib.oz2o_mod_i64.argtypes = [i64, P, i32, P]
        _lib.oz2o_crt.argtypes = [i64, i32, P, P, P, d, d, d, i32, i32, P, P, P, P]
        _lib.oz2o_unscale.argtypes = [i32, i32, P, P, P, i32, P]
        _lib.oz2o_log2f.argtypes = [i64, P, P]
        _lib.oz2o_exact_residual.argtypes = [i32, i32, i32, P, i64, i64, P, i64, i64, P, P]
        _lib.oz2o_exact_abs_sums.argtypes = [i32, i32, P, i64, i64, P]
        _lib.oz2o_num_threads.restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _strides(X: np.ndarray):
    return X.strides[0] // X.itemsize, X.strides[1] // X.itemsize


INT32_MIN = -(1 << 31)


# --------------------------------------------------------------------------- #
# Small elementwise helpers (exact)
# --------------------------------------------------------------------------- #
def floor_log2_absmax(X: np.ndarray, axis: int) -> np.ndarray:
    """floor(log2 max |x|) along `axis` (alpha_i / beta_j of Theorem 2); INT32_MIN if zero."""
    X = np.asarray(X, dtype=np.float64)
    V = X if axis == 1 else X.T
    out = np.empty(V.shape[0], dtype=np.int32)
    rs, cs = _strides(V)
    lib().oz2o_floor_log2_absmax(V.shape[0], V.shape[1], _p(V), rs, cs, _p(out))
    return out


def single_up(v: np.ndarray) -> np.ndarray:
    """single_up(.) of nonnegative integers below 2^31 (Algorithm 2, Dbar)."""
    v = np.asarray(v, dtype=np.float64)
    f = v.astype(np.float32)
    low = f.astype(np.float64) < v
    f[low] = np.nextafter(f[low], np.float32(np.inf))
    return f


def log2f(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    lib().oz2o_log2f(x.size, _p(x), _p(out))
    return out


def exponent_shift(c: np.float32, e: np.ndarray, Pprime: np.float32) -> np.ndarray:
    """floor(fl_down(fma(c, e, P'))) of Algorithm 2 = floor(c*e + P') exactly.

    c and e are FP32, so c*e has at most 48 significant bits and |c*e| < 16;
    P' < 200 is a multiple of 2^-16 at worst.  The sum therefore fits the 53
    bits of FP64 and both operations below are exact.
    """
    v = np.float64(c) * e.astype(np.float64) + np.float64(Pprime)
    return np.floor(v).astype(np.int64)


# --------------------------------------------------------------------------- #
# Algorithm 2: Scaling
# --------------------------------------------------------------------------- #
def ceil_sqrt(x: int) -> int:
    """ceil(sqrt(x)) of a nonnegative integer, exactly."""
    r = math.isqrt(x)
    return r if r * r == x else r + 1


def fast_cbar_maxima(Abar: np.ndarray, Bbar: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Fast mode (reading; the paper only names the mode): row and column maxima
    of the Cauchy-Schwarz majorant chat_ij = ceil(||Abar_i||_2 ||Bbar_j||_2) >= cbar_ij,
    i.e. ceil(sqrt(ssA_i * max_j ssB_j)) and ceil(sqrt(max_i ssA_i * ssB_j)), with
    ssA_i = sum_h abar_ih^2 and ssB_j = sum_h bbar_hj^2 exact integers."""
    ssA = [int(v) for v in (Abar.astype(np.int64) ** 2).sum(axis=1)]
    ssB = [int(v) for v in (Bbar.astype(np.int64) ** 2).sum(axis=0)]
    mA = max(ssA, default=0)
    mB = max(ssB, default=0)
    row = np.array([ceil_sqrt(a * mB) for a in ssA], dtype=np.int64)
    col = np.array([ceil_sqrt(mA * b) for b in ssB], dtype=np.int64)
    return row, col


def scaling(A: np.ndarray, B: np.ndarray, N: int, b: int = 64,
            mu_in: np.ndarray | None = None, nu_in: np.ndarray | None = None, fast: bool = False) -> dict:
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    C = constants(N, b)
    L = lib()
    # mu'_i = 5 - floor(log2 max_h |a_ih|); nu'_j likewise (eq. mu'nu')
    alpha = floor_log2_absmax(A, axis=1)
    beta = floor_log2_absmax(B, axis=0)
    mu_p = np.where(alpha == INT32_MIN, 0, 5 - alpha.astype(np.int64)).astype(np.int32)
    nu_p = np.where(beta == INT32_MIN, 0, 5 - beta.astype(np.int64)).astype(np.int32)
    # Abar = ceil(diag(2^mu') |A|), Bbar = ceil(|B| diag(2^nu'))
    Abar = np.empty((m, k), dtype=np.int8)
    rs, cs = _strides(A)
    L.oz2o_ceil_scaled_abs(m, k, _p(A), rs, cs, _p(mu_p), _p(Abar))
    BbarT = np.empty((n, k), dtype=np.int8)
    BT = B.T
    rs, cs = _strides(BT)
    L.oz2o_ceil_scaled_abs(n, k, _p(BT), rs, cs, _p(nu_p), _p(BbarT))
    Bbar = np.ascontiguousarray(BbarT.T)
    if not fast:
        # Cbar = Abar Bbar, exact
        Cbar = gemm_i8(Abar, Bbar)
        cmax_row = Cbar.max(axis=1) if n else np.zeros(m, np.int64)
        cmax_col = Cbar.max(axis=0) if m else np.zeros(n, np.int64)
        # Dbar = single_up(Cbar); e_i = log2f(max_h dbar_ih); f_j = log2f(max_h dbar_hj)
        Dbar = single_up(Cbar)
        drow = Dbar.max(axis=1) if n > 0 else np.zeros(m, np.float32)
        dcol = Dbar.max(axis=0) if m > 0 else np.zeros(n, np.float32)
    else:
        Cbar = None
        cmax_row, cmax_col = fast_cbar_maxima(Abar, Bbar)
        drow = single_up(cmax_row)
        dcol = single_up(cmax_col)
    drow = np.where(drow == 0, np.float32(1), drow)          # reading: empty row -> 1
    dcol = np.where(dcol == 0, np.float32(1), dcol)
    e = log2f(drow)
    f = log2f(dcol)
    mu = (mu_p + exponent_shift(C.c, e, C.Pprime)).astype(np.int32)
    nu = (nu_p + exponent_shift(C.c, f, C.Pprime)).astype(np.int32)
    own_mu, own_nu = mu, nu
    if mu_in is not None:
        mu = np.asarray(mu_in, dtype=np.int32)
    if nu_in is not None:
        nu = np.asarray(nu_in, dtype=np.int32)
    # A' = trunc(diag(2^mu) A), B' = trunc(B diag(2^nu))
    Ap = trunc_scaled_rows(A, mu)
    Bp = np.ascontiguousarray(trunc_scaled_rows(B.T, nu).T)
    return dict(alpha=alpha, beta=beta, mu_p=mu_p, nu_p=nu_p, Abar=Abar, Bbar=Bbar,
                Cbar=Cbar, cmax_row=cmax_row, cmax_col=cmax_col,
                e=e, f=f, mu=mu, nu=nu, own_mu=own_mu, own_nu=own_nu, Ap=Ap, Bp=Bp)


def trunc_scaled_rows(X: np.ndarray, shift: np.ndarray) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    rows, cols = X.shape
    out = np.empty((rows, cols), dtype=np.float64)
    rs, cs = _strides(X)
    sh = np.ascontiguousarray(shift, dtype=np.int32)
    lib().oz2o_trunc_scaled(rows, cols, _p(X), rs, cs, _p(sh), _p(out))
    return out


def gemm_i8(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.int8)
    Y = np.ascontiguousarray(Y, dtype=np.int8)
    m, k = X.shape
    n = Y.shape[1]
    Z = np.empty((m, n), dtype=np.int64)
    lib().oz2o_gemm_i8_i64(m, n, k, _p(X), _p(Y), _p(Z))
    return Z


def residues(X: np.ndarray, p: int) -> np.ndarray:
    """mod(X, p) of Algorithm 3 as INT8 (X integer-valued doubles)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.empty(X.shape, dtype=np.int8)
    lib().oz2o_residues(X.size, _p(X), p, _p(out))
    return out


def mod_i64(X: np.ndarray, p: int) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.int64)
    out = np.empty(X.shape, dtype=np.int8)
    lib().oz2o_mod_i64(X.size, _p(X), p, _p(out))
    return out


# --------------------------------------------------------------------------- #
# Algorithm 3: CRT
# --------------------------------------------------------------------------- #
def crt(Ap: np.ndarray, Bp: np.ndarray, N: int, b: int = 64, keep_residues: bool = False,
        consts=None, fma_chain: bool = False) -> dict:
    C = consts if consts is not None else constants(N, b)
    m, k = Ap.shape
    n = Bp.shape[1]
    W = np.empty((N, m, n), dtype=np.int8)
    Ares = np.empty((N, m, k), dtype=np.int8) if keep_residues else None
    Bres = np.empty((N, k, n), dtype=np.int8) if keep_residues else None
    for l, pl in enumerate(C.p):
        Al = residues(Ap, pl)                 # A'_l = mod(A', p_l)
        Bl = residues(Bp, pl)                 # B'_l = mod(B', p_l)
        if keep_residues:
            Ares[l], Bres[l] = Al, Bl
        W[l] = mod_i64(gemm_i8(Al, Bl), pl)   # W_l = mod(A'_l B'_l, p_l)
    out = crt_from_W(W, N, b, consts=C, fma_chain=fma_chain)
    out.update(W=W, Ares=Ares, Bres=Bres)
    return out


def crt_from_W(W: np.ndarray, N: int, b: int = 64, consts=None, fma_chain: bool = False) -> dict:
    """Algorithm 3 from W_l on; `consts` replaces the tables (tests plant mistakes with it).

    C'(1), C'(2) are the exactly rounded sums; fma_chain=True takes them as fma
    chains in ascending l instead (the other reading of fl(sum))."""
    C = consts if consts is not None else constants(N, b)
    shape = W.shape[1:]
    count = int(np.prod(shape))
    W = np.ascontiguousarray(W, dtype=np.int8)
    s1 = np.array(C.s1, dtype=np.float64)
    s2 = np.array(C.s2, dtype=np.float64)
    C1 = np.empty(count); C2 = np.empty(count); Q = np.empty(count); Cpp = np.empty(count)
    lib().oz2o_crt(count, N, _p(W), _p(s1), _p(s2), C.P1, C.P2, C.Pinv, b, int(fma_chain),
                   _p(C1), _p(C2), _p(Q), _p(Cpp))
    return dict(C1=C1.reshape(shape), C2=C2.reshape(shape), Q=Q.reshape(shape),
                Cpp=Cpp.reshape(shape))


def unscale(Cpp: np.ndarray, mu: np.ndarray, nu: np.ndarray, b: int = 64) -> np.ndarray:
    Cpp = np.ascontiguousarray(Cpp, dtype=np.float64)
    m, n = Cpp.shape
    out = np.empty((m, n), dtype=np.float64)
    lib().oz2o_unscale(m, n, _p(Cpp), _p(np.ascontiguousarray(mu, np.int32)),
                       _p(np.ascontiguousarray(nu, np.int32)), b, _p(out))
    return out if b == 64 else out.astype(np.float32)


# --------------------------------------------------------------------------- #
# Algorithm 1: OS_II
# --------------------------------------------------------------------------- #
def os_ii(A: np.ndarray, B: np.ndarray, N: int, b: int = 64,
          mu_in=None, nu_in=None, keep_residues: bool = False, consts=None, fast: bool = False,
          fma_chain: bool = False) -> dict:
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if not (N_MIN <= N <= N_MAX):
        raise ValueError("N out of range")
    if A.shape[1] > K_MAX:
        raise ValueError("k > 2^17")
    s = scaling(A, B, N, b, mu_in, nu_in, fast=fast)
    r = crt(s["Ap"], s["Bp"], N, b, keep_residues, consts, fma_chain)
    s.update(r)
    s["C"] = unscale(r["Cpp"], s["mu"], s["nu"], b)
    s["N"], s["b"] = N, b
    return s


# --------------------------------------------------------------------------- #
# Split-K beyond k = 2^17 (an extension; the paper assumes k <= 2^17)
# --------------------------------------------------------------------------- #
def splitk_ranges(k: int) -> list[tuple[int, int]]:
    """Consecutive K ranges [k0, k1): S = ceil(k / 2^17) are wanted, each of
    kc = 64 ceil(ceil(k / S) / 64) <= 2^17 values except a shorter last one."""
    if k <= K_MAX:
        return [(0, k)]
    S = -(-k // K_MAX)
    kc = 64 * -(-(-(-k // S)) // 64)
    return [(k0, min(k, k0 + kc)) for k0 in range(0, k, kc)]


def os_ii_splitk(A: np.ndarray, B: np.ndarray, N, b: int = 64, mu_in=None, nu_in=None,
                 fast: bool = False) -> dict:
    """C = sum over the K ranges of OS_II(A[:, range], B[range, :]), added in
    range order in the output precision (FP64 for b = 64, FP32 for b = 32).

    N: one int for every range or a list with one per range; mu_in / nu_in:
    lists with one vector per range (or None).  Returns C, the per-range
    results ("parts") and the running sums after each addition ("partial")."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    ranges = splitk_ranges(A.shape[1])
    Ns = list(N) if isinstance(N, (list, tuple, np.ndarray)) else [int(N)] * len(ranges)
    parts, partial, C = [], [], None
    for s, (k0, k1) in enumerate(ranges):
        r = os_ii(np.ascontiguousarray(A[:, k0:k1]), np.ascontiguousarray(B[k0:k1]), int(Ns[s]), b,
                  mu_in=None if mu_in is None else mu_in[s], nu_in=None if nu_in is None else nu_in[s],
                  fast=fast)
        C = r["C"].copy() if C is None else C + r["C"]   # one rounding per addition
        parts.append(r)
        partial.append(C.copy())
    return dict(C=C, parts=parts, partial=partial, ranges=ranges)


def bound_splitk(A: np.ndarray, B: np.ndarray, res: dict, b: int = 64) -> np.ndarray:
    """Upper bound of |AB - C| for os_ii_splitk's result: the sum of the ranges'
    bounds (from their exponents) plus u |running sum| for every addition, and
    half the smallest subnormal per range for underflow."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    u = 2.0 ** -53 if b == 64 else 2.0 ** -24
    eta = 2.0 ** -1075 if b == 64 else 2.0 ** -150
    total = np.zeros((A.shape[0], B.shape[1]))
    for s, ((k0, k1), r) in enumerate(zip(res["ranges"], res["parts"])):
        As, Bs = A[:, k0:k1], B[k0:k1]
        total += bound_from_exponents(As, Bs, r["mu"], r["nu"], r["Ap"], r["Bp"], r["N"], b) + eta
        if s > 0:
            total += u * np.abs(res["partial"][s].astype(np.float64)) + eta
    return total * _UP


# --------------------------------------------------------------------------- #
# Complex products (an extension; the paper's analysis covers real GEMM)
# --------------------------------------------------------------------------- #
def complex_parts(A: np.ndarray, B: np.ndarray):
    """The real operands of a complex product A B (A m x k, B k x n complex):
    A_s = [Re A, Im A] (m x 2k), B_1 = [Re B; -Im B], B_2 = [Im B; Re B] (2k x n),
    so that A_s B_1 = Re(A B) and A_s B_2 = Im(A B) exactly."""
    A = np.asarray(A)
    B = np.asarray(B)
    As = np.hstack([A.real, A.imag]).astype(np.float64)
    B1 = np.vstack([B.real, -B.imag]).astype(np.float64)
    B2 = np.vstack([B.imag, B.real]).astype(np.float64)
    return As, B1, B2


def os_ii_complex(A: np.ndarray, B: np.ndarray, N, b: int = 64, mu_in=None, nu_in=None,
                  fast: bool = False) -> dict:
    """C = A B for complex A, B (already transposed / conjugated as wanted) as
    two real emulated products over 2k (split-K when 2k > 2^17).  N: an int,
    or a pair (one per part) of ints or per-range lists; mu_in / nu_in: a pair
    of per-range lists or None."""
    As, B1, B2 = complex_parts(A, B)
    Ns = N if isinstance(N, (list, tuple)) else (N, N)
    parts = []
    for p, Bp in enumerate((B1, B2)):
        parts.append(os_ii_splitk(As, Bp, Ns[p], b, mu_in=None if mu_in is None else mu_in[p],
                                  nu_in=None if nu_in is None else nu_in[p], fast=fast))
    dt = np.complex128 if b == 64 else np.complex64
    C = np.empty(parts[0]["C"].shape, dtype=dt)
    C.real, C.imag = parts[0]["C"], parts[1]["C"]
    return dict(C=C, parts=parts, As=As, B1=B1, B2=B2)


def os_ii_block(A_rows: np.ndarray, B_cols: np.ndarray, mu: np.ndarray, nu: np.ndarray,
                N: int, b: int = 64) -> np.ndarray:
    """Entries C_ij for the given rows of A and columns of B with injected mu, nu.

    Algorithm 2 only fixes mu and nu; once they are given, each entry depends on
    row i of A and column j of B alone (A' rows, B' columns, Algorithm 3 and the
    final scaling), so sampled entries of a large product can be checked one by one.
    """
    Ap = trunc_scaled_rows(A_rows, mu)
    Bp = np.ascontiguousarray(trunc_scaled_rows(np.asarray(B_cols, np.float64).T, nu).T)
    r = crt(Ap, Bp, N, b)
    return unscale(r["Cpp"], mu, nu, b)


# --------------------------------------------------------------------------- #
# Exact products, errors and the bounds of Theorem 2
# --------------------------------------------------------------------------- #
def exact_residual(X: np.ndarray, Y: np.ndarray, Cm: np.ndarray | None = None) -> np.ndarray:
    """RN(X Y - Cm), computed exactly and rounded once (X m x k, Y k x n doubles)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    m, k = X.shape
    n = Y.shape[1]
    out = np.empty((m, n), dtype=np.float64)
    xr, xc = _strides(X)
    yr, yc = _strides(Y)
    Cm = None if Cm is None else np.ascontiguousarray(Cm, dtype=np.float64)
    lib().oz2o_exact_residual(m, n, k, _p(X), xr, xc, _p(Y), yr, yc, _p(Cm), _p(out))
    return out


def exact_product(A, B):
    return exact_residual(A, B, None)


def abs_sums(X: np.ndarray, axis: int) -> np.ndarray:
    """Correctly rounded sum_h |x| along `axis`."""
    X = np.asarray(X, dtype=np.float64)
    V = X if axis == 1 else X.T
    out = np.empty(V.shape[0])
    rs, cs = _strides(V)
    lib().oz2o_exact_abs_sums(V.shape[0], V.shape[1], _p(V), rs, cs, _p(out))
    return out


_UP = 1.0 + 2.0 ** -40


def pow2_prime(alpha: np.ndarray, cmax: np.ndarray) -> np.ndarray:
    """2^alpha' = 2^alpha * sqrt(max cbar) (Theorem 2), rounded up; 0 for empty rows."""
    out = np.zeros(alpha.shape[0])
    ok = (alpha != INT32_MIN) & (cmax > 0)
    out[ok] = np.ldexp(np.sqrt(cmax[ok].astype(np.float64)), alpha[ok]) * _UP
    return out


def bounds(A: np.ndarray, B: np.ndarray, res: dict) -> tuple[np.ndarray, np.ndarray]:
    """Upper bounds of |AB - C| per entry: eq. thm:err-1 and eq. thm:err-2."""
    N, b = res["N"], res["b"]
    k = A.shape[1]
    bt = bound_terms(N, b)
    t = bt["t"]
    R = abs_sums(A, axis=1) * _UP            # |A| v
    K = abs_sums(B, axis=0) * _UP            # v^T |B|
    a2 = pow2_prime(res["alpha"], res["cmax_row"])
    b2 = pow2_prime(res["beta"], res["cmax_col"])
    absApBp = np.abs(exact_residual(res["Ap"], res["Bp"])) * _UP
    common = t * np.outer(R, b2) + t * np.outer(a2, K)
    t2ab = (t * t) * np.outer(a2, b2)
    err1 = (common + (k + bt["gN"] + bt["h"] * absApBp) * t2ab) * _UP
    err2 = (common + (k + bt["rb"]) * t2ab) * _UP
    return err1, err2


# --------------------------------------------------------------------------- #
# Exponent checks against the paper's definitions
# --------------------------------------------------------------------------- #
def mu_band(mu_p: np.ndarray, cmax: np.ndarray, N: int, b: int = 64) -> tuple[np.ndarray, np.ndarray]:
    """Range of mu allowed by Algorithm 2 under assumption (1) on log2f.

    With d = max dbar (1 for an empty row), any FP32 e with
    |e - log2 d| <= 4 u32 log2 d gives mu = mu' + floor(c e + P'); c < 0 makes
    this non-increasing in e, so the extremes come from the smallest and the
    largest admissible FP32 e.
    """
    C = constants(N, b)
    d = single_up(cmax).astype(np.float64)
    d = np.where(d == 0, 1.0, d)
    lo = np.empty(len(d), np.int64)
    hi = np.empty(len(d), np.int64)
    u4 = 4 * float(U32)
    for i, di in enumerate(d):
        lg = math.log2(di)
        e_lo = np.float32(lg * (1 - u4))
        if float(e_lo) < lg * (1 - u4) * (1 - 1e-15):
            e_lo = np.nextafter(e_lo, np.float32(np.inf))
        e_hi = np.float32(lg * (1 + u4))
        if float(e_hi) > lg * (1 + u4) * (1 + 1e-15):
            e_hi = np.nextafter(e_hi, np.float32(-np.inf))
        if lg == 0.0:
            e_lo = e_hi = np.float32(0.0)
        hi[i] = exponent_shift(C.c, np.array([e_lo], np.float32), C.Pprime)[0]
        lo[i] = exponent_shift(C.c, np.array([e_hi], np.float32), C.Pprime)[0]
    return mu_p + lo, mu_p + hi


# --------------------------------------------------------------------------- #
# Bound-chosen N (a reading: the paper motivates choosing N from the bound
# for a target accuracy but gives no rule; this takes the smallest N whose
# N-dependent part of eq. thm:err-2 meets the target)
# --------------------------------------------------------------------------- #
def choose_N(A: np.ndarray, B: np.ndarray, alpha, beta, cmax_row, cmax_col,
             tau: float, nmax: int, b: int = 64) -> tuple[int, dict]:
    """Smallest N in [2, nmax] whose N-dependent part of eq. thm:err-2 is <= tau * L.

    T_N = t (max_i R_i)(max_j 2^beta'_j) + t (max_i 2^alpha'_i)(max_j K_j)
          + (k + g_N) t^2 (max_i 2^alpha'_i)(max_j 2^beta'_j)
    with R = |A| v, K = v^T |B|, g_N the P-proportional part of R_b (Lemma 4),
    and L = max_h (max_i |a_ih|)(max_j |b_hj|), a lower bound of
    max_ij (|A||B|)_ij.  Every maximum of a sum of nonnegative terms is bounded
    by the sum of the maxima, so T_N bounds the N-dependent part of the bound
    on every entry.  Returns (N, info); nmax when no N qualifies.
    """
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    m, k = A.shape
    n = B.shape[1]
    R = abs_sums(A, 1)
    K = abs_sums(B, 0)
    a2 = pow2_prime(np.asarray(alpha), np.asarray(cmax_row))
    b2 = pow2_prime(np.asarray(beta), np.asarray(cmax_col))
    L = float(np.max(np.abs(A).max(axis=0) * np.abs(B).max(axis=1))) if m and n and k else 0.0
    return choose_N_from_maxima(float(R.max(initial=0)), float(K.max(initial=0)), float(a2.max(initial=0)),
                                float(b2.max(initial=0)), L, k, tau, nmax, b)


def choose_N_from_maxima(maxR: float, maxK: float, ma2: float, mb2: float, L: float, k: int,
                         tau: float, nmax: int, b: int = 64) -> tuple[int, dict]:
    """The N rule of choose_N from its five maxima (max_i R_i, max_j K_j,
    max_i 2^alpha'_i, max_j 2^beta'_j, L) and k."""
    chosen, ratios = nmax, {}
    for N in range(N_MIN, nmax + 1):
        bt = bound_terms(N, b)
        t = bt["t"]
        T = t * (maxR * mb2 + ma2 * maxK) + (k + bt["gN"]) * t * t * ma2 * mb2
        ratios[N] = T / L if L > 0 else 0.0
    for N in range(N_MIN, nmax + 1):
        if ratios[N] <= tau:
            chosen = N
            break
    return chosen, dict(L=L, ratios=ratios, maxR=maxR, maxK=maxK, max2a=ma2, max2b=mb2)


# --------------------------------------------------------------------------- #
# Componentwise N rule (a reading: Theorem 2 bounds every entry; this rule
# asks the N-dependent part of eq. thm:err-1 to meet the target relative to
# (|A||B|)_ij on every entry instead of relative to max (|A||B|))
# --------------------------------------------------------------------------- #
def floor_scaled_abs(X: np.ndarray, shift: np.ndarray, axis: int) -> np.ndarray:
    """floor(2^shift |x|) with the shift of each row (axis = 1) or column
    (axis = 0): nonnegative integers <= 63 for shift = 5 - floor(log2 max)."""
    X = np.abs(np.asarray(X, np.float64))
    sh = np.asarray(shift, np.int64)
    sc = np.ldexp(X, sh[:, None] if axis == 1 else sh[None, :])     # exact (or 0 on underflow)
    return np.floor(sc).astype(np.int8)


def componentwise_lower(A: np.ndarray, B: np.ndarray, mu_p: np.ndarray, nu_p: np.ndarray) -> np.ndarray:
    """L_ij = 2^-(mu'_i + nu'_j) (Ahat Bhat)_ij <= (|A||B|)_ij, Ahat = floor(2^mu' |A|),
    Bhat = floor(|B| 2^nu'): every term of Ahat Bhat is at most the scaled |a_ih||b_hj|."""
    Ch = gemm_i8(floor_scaled_abs(A, mu_p, 1), floor_scaled_abs(B, nu_p, 0)).astype(np.float64)
    return np.ldexp(Ch, -(np.asarray(mu_p, np.int64)[:, None] + np.asarray(nu_p, np.int64)[None, :]))


def componentwise_maxima(A: np.ndarray, B: np.ndarray, alpha, beta, cmax_row, cmax_col):
    """max_ij X_ij / L_ij and max_ij Y_ij / L_ij (upper bounds), where
    X_ij = R_i 2^beta'_j + 2^alpha'_i K_j and Y_ij = 2^alpha'_i 2^beta'_j multiply
    t and t^2 in the N-dependent part of eq. thm:err-1 (R = |A|v, K = v^T|B|),
    and L_ij is componentwise_lower.  An entry with L_ij = 0 gives +inf."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    alpha = np.asarray(alpha)
    beta = np.asarray(beta)
    mu_p = np.where(alpha == INT32_MIN, 0, 5 - alpha.astype(np.int64))
    nu_p = np.where(beta == INT32_MIN, 0, 5 - beta.astype(np.int64))
    R = abs_sums(A, 1) * _UP
    K = abs_sums(B, 0) * _UP
    a2 = pow2_prime(alpha, np.asarray(cmax_row))
    b2 = pow2_prime(beta, np.asarray(cmax_col))
    L = componentwise_lower(A, B, mu_p, nu_p)
    X = (np.outer(R, b2) + np.outer(a2, K)) * _UP
    Y = np.outer(a2, b2) * _UP
    # entries with X = Y = 0 (a zero row of A or column of B) need no protection
    live = (X > 0) | (Y > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        x = np.where(live, np.where(L > 0, X / L, np.inf), 0.0) * _UP
        y = np.where(live, np.where(L > 0, Y / L, np.inf), 0.0) * _UP
    return float(x.max(initial=0.0)), float(y.max(initial=0.0))


def choose_N_componentwise(A: np.ndarray, B: np.ndarray, alpha, beta, cmax_row, cmax_col,
                           tau: float, nmax: int, b: int = 64) -> tuple[int, dict]:
    """Smallest N in [2, nmax] with t_N xmax + (k + g_N) t_N^2 ymax <= tau
    (componentwise_maxima), i.e. the N-dependent part of eq. thm:err-1 is at most
    tau (|A||B|)_ij on every entry; nmax when no N qualifies."""
    k = np.asarray(A).shape[1]
    xmax, ymax = componentwise_maxima(A, B, alpha, beta, cmax_row, cmax_col)
    chosen, ratios = nmax, {}
    for N in range(N_MIN, nmax + 1):
        bt = bound_terms(N, b)
        t = bt["t"]
        ratios[N] = t * xmax + (k + bt["gN"]) * t * t * ymax if np.isfinite(xmax) and np.isfinite(ymax) \
            else np.inf
    for N in range(N_MIN, nmax + 1):
        if ratios[N] <= tau:
            chosen = N
            break
    return chosen, dict(ratios=ratios, xmax=xmax, ymax=ymax)


# --------------------------------------------------------------------------- #
# Exact integer checks (Lemmas 0, 2, 3; Theorem 1)
# --------------------------------------------------------------------------- #
def crt_exact(W: np.ndarray, N: int) -> tuple[list, list]:
    """A'B' = mod(sum_l P/p_l q_l W_l, P) (Lemma 3 proof) and Q_exact, as Python ints."""
    C = constants(N, 64)
    P = C.P
    flat = W.reshape(N, -1)
    AB, Qx = [], []
    for e in range(flat.shape[1]):
        S = sum(int(x) * int(w) for x, w in zip(C.x, flat[:, e]))
        q = (2 * S + P) // (2 * P)            # round(S/P); ties cannot occur (Lemma 3)
        AB.append(S - P * q)
        Qx.append(q)
    return AB, Qx


def ozaki_exponent_floor_ok(mu, alpha, cmax, N) -> np.ndarray:
    """Lemma 1, eq. (mu_i lower bound): 2^(2 mu_i + 2 alpha_i - 5) * max cbar_i >= P - 1."""
    P = constants(N, 64).P
    ok = []
    for mi, ai, ci in zip(mu, alpha, cmax):
        if ai == INT32_MIN or ci == 0:
            ok.append(True)
            continue
        ex = 2 * int(mi) + 2 * int(ai) - 5
        lhs = Fraction(int(ci)) * (Fraction(2) ** ex)
        ok.append(lhs >= P - 1)
    return np.array(ok)


def bound_from_exponents(A_rows: np.ndarray, B_cols: np.ndarray, mu: np.ndarray, nu: np.ndarray,
                         Ap_rows: np.ndarray, Bp_cols: np.ndarray, N: int, b: int = 64) -> np.ndarray:
    """Upper bound of |AB - C| per entry given the exponents actually used.

    The proof of Lemma 1 bounds the truncation error with |Delta_A|, |Delta_B| < 1:
      |AB - 2^-mu A'B' 2^-nu| <= 2^-nu_j (|A| v)_i + 2^-mu_i (v^T |B|)_j + k 2^-(mu_i+nu_j),
    and Lemma 4 adds 2^-(mu_i+nu_j) R_b.  Valid whenever Lemma 0 holds for the
    entries (checked separately), so it applies to injected exponents too.
    """
    A_rows = np.asarray(A_rows, np.float64)
    B_cols = np.asarray(B_cols, np.float64)
    k = A_rows.shape[1]
    bt = bound_terms(N, b)
    R = abs_sums(A_rows, 1) * _UP
    K = abs_sums(B_cols, 0) * _UP
    absApBp = np.abs(exact_residual(Ap_rows, Bp_cols)) * _UP
    smu = np.ldexp(1.0, -np.asarray(mu, np.int64))
    snu = np.ldexp(1.0, -np.asarray(nu, np.int64))
    Rb = bt["gN"] + bt["h"] * absApBp
    return (np.outer(R, snu) + np.outer(smu, K) + (k + Rb) * np.outer(smu, snu)) * _UP


def lemma0_holds(Ap_rows: np.ndarray, Bp_cols: np.ndarray, N: int) -> bool:
    """Lemma 0: |A'||B'| < P/2 on every entry (FP64 upper bound, exact fallback)."""
    P = constants(N, 64).P
    ub = exact_product(np.abs(Ap_rows), np.abs(Bp_cols)) * (1 + 2.0 ** -40)
    if (ub < float(P) / 2 * (1 - 2.0 ** -40)).all():
        return True
    IA = [[int(v) for v in row] for row in np.abs(Ap_rows)]
    IB = [[int(v) for v in col] for col in np.abs(Bp_cols).T]
    return all(2 * sum(a * b for a, b in zip(ra, cb)) < P for ra in IA for cb in IB)
