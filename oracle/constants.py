"""Exact constants of the Ozaki-II scheme, computed with Python integers and rationals.

TEST INFRASTRUCTURE ONLY.  This module belongs to the CPU oracle: only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The GPU library generates its own tables independently.

Sources (arXiv 2602.02549, "Error Analysis of Matrix Multiplication Emulation
Using Ozaki-II Scheme"):
  * Theorem 1 (CRT) and Step 1 of Section 2.2: P, q_l with q_l < p_l.
  * Section 3.1, eq. (p_list): the fixed list of 49 pairwise-coprime moduli.
  * Section 3.1: P1 = double(P), P2 = double(P - P1) (DGEMM) or 0 (SGEMM);
    s_l1 keeps the upper beta_l bits of P/p_l*q_l, s_l2 = double(rest) (DGEMM);
    s_l1 = double(P/p_l*q_l), s_l2 = 0 (SGEMM).
  * Algorithm 2, first line: P' = single_down(log2(P-1)/2 - 0.5).
  * Algorithm 2, mu/nu lines: c = single_down(-0.5/(1-4*u32)).
  * Algorithm 3: P_inv = double(1/P).
  * Theorem 2 / Lemma 4: t = 1/sqrt(2^5 (P-1)), rho = sum floor(p_l/2).
  * Proof of Lemma 0: the exhaustive evaluation behind the constant 2^-21
    (lemma0_margin).

Reading taken where the paper's Figure 1 is missing: "retains only the upper
beta_l bits" is truncation toward zero onto the grid
g = 2^(ceil(log2 rho) + floor(log2 r) - 52), r = max_l P/p_l*q_l (the proof
of Lemma 2 uses 0 <= P/p_l*q_l - s_l1 and s_l1 in g*Z).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from decimal import Decimal, localcontext
from fractions import Fraction
from functools import lru_cache

import numpy as np

# Section 3.1, eq. (p_list): the moduli in the order used; N takes the first N.
MODULI = (256, 255, 253, 251, 247, 241, 239, 233, 229, 227,
          223, 217, 211, 199, 197, 193, 191, 181, 179, 173,
          167, 163, 157, 151, 149, 139, 137, 131, 127, 113,
          109, 107, 103, 101, 97, 89, 83, 79, 73, 71,
          67, 61, 59, 53, 47, 43, 41, 37, 29)

N_MIN, N_MAX = 2, 49
K_MAX = 1 << 17          # Section 3: k <= 2^17
U32 = Fraction(1, 1 << 24)
U64 = Fraction(1, 1 << 53)


def ceil_log2_int(x: int) -> int:
    """ceil(log2 x) for a positive integer, exactly."""
    return (x - 1).bit_length()


def floor_log2_int(x: int) -> int:
    """floor(log2 x) for a positive integer, exactly."""
    return x.bit_length() - 1


def f32_round_down(v: Fraction) -> np.float32:
    """single_down(v): the largest FP32 number <= v (v exact rational)."""
    f = np.float32(float(v))
    ninf, pinf = np.float32(-np.inf), np.float32(np.inf)
    while Fraction(float(f)) > v:
        f = np.nextafter(f, ninf)
    while Fraction(float(np.nextafter(f, pinf))) <= v:
        f = np.nextafter(f, pinf)
    return f


def log2_decimal(x: int, digits: int = 80) -> Decimal:
    """log2 of a positive integer to `digits` significant digits."""
    with localcontext() as ctx:
        ctx.prec = digits + 10
        return Decimal(x).ln() / Decimal(2).ln()


@dataclass(frozen=True)
class Constants:
    N: int
    b: int                      # 64 (DGEMM) or 32 (SGEMM)
    p: tuple                    # first N moduli
    P: int
    q: tuple                    # q_l = (P/p_l)^(-1) mod p_l
    x: tuple                    # P/p_l * q_l (exact integers)
    rho: int
    s1: tuple                   # doubles
    s2: tuple                   # doubles
    g: Fraction                 # grid of s1 (DGEMM); 0 for SGEMM
    P1: float
    P2: float
    Pinv: float
    Pprime: np.float32
    c: np.float32

    @property
    def t(self) -> float:
        """t = 1/sqrt(2^5 (P-1)) (Theorem 2), rounded up slightly for use in bounds."""
        return t_upper(self.P)


def t_upper(P: int) -> float:
    """An FP64 upper bound of 1/sqrt(32 (P-1)) (relative slack ~2^-50)."""
    v = 1.0 / math.sqrt(32.0 * float(P - 1))
    return v * (1.0 + 2.0 ** -50)


@lru_cache(maxsize=None)
def constants(N: int, b: int = 64) -> Constants:
    if not (N_MIN <= N <= N_MAX):
        raise ValueError("N must be in [2, 49]")
    if b not in (32, 64):
        raise ValueError("b must be 32 or 64")
    p = MODULI[:N]
    P = math.prod(p)
    q = tuple(pow(P // pl, -1, pl) for pl in p)          # Theorem 1
    x = tuple((P // pl) * ql for pl, ql in zip(p, q))
    rho = sum(pl // 2 for pl in p)
    r = max(x)
    if b == 64:
        e = ceil_log2_int(rho) + floor_log2_int(r) - 52
        g = Fraction(2) ** e
        s1f = [Fraction(math.floor(Fraction(xl) / g)) * g for xl in x]
        s1 = tuple(float(v) for v in s1f)
        assert all(Fraction(a) == v for a, v in zip(s1, s1f))   # representable
        s2 = tuple(float(Fraction(xl) - v) for xl, v in zip(x, s1f))
        P1 = float(P)
        P2 = float(P - int(P1))
    else:
        g = Fraction(0)
        s1 = tuple(float(xl) for xl in x)
        s2 = tuple(0.0 for _ in x)
        P1 = float(P)
        P2 = 0.0
    Pinv = float(Fraction(1, P))
    lg = log2_decimal(P - 1)
    v = Fraction(lg / 2 - Decimal("0.5"))
    Pprime = f32_round_down(v)
    # the decimal approximation is far closer than any FP32 spacing near P'
    assert abs(Fraction(float(Pprime)) - v) > Fraction(1, 10 ** 40)
    c = f32_round_down(Fraction(-1, 2) / (1 - 4 * U32))
    return Constants(N, b, p, P, q, x, rho, s1, s2, g, P1, P2, Pinv, Pprime, c)


def bound_terms(N: int, b: int = 64) -> dict:
    """Scalars of Theorem 2 (eq. thm:err-1 / thm:err-2) and Lemma 4 for N moduli.

    Returns FP64 upper bounds of
      t, g_N (the P-proportional part of R_b), h_b (coefficient of |A'B'| in R_b),
      r_b (eq. thm:err-2), each as a Python float rounded up by a 2^-40 factor.
    """
    C = constants(N, b)
    P, rho = C.P, C.rho
    up = 1 + Fraction(1, 1 << 40)
    if b == 64:
        gN = (1 + 3 * U64) * Fraction(2) ** (1 + ceil_log2_int(rho)) * (N + 2) * U64 ** 2 * rho * P
        h = 3 * U64
        rb = gN + Fraction(3, 2) * U64 * P
    else:
        gN = (1 + U32) * (N + 2) * U64 * rho * P
        h = U32
        rb = gN + Fraction(1, 2) * U32 * P
    return {"t": C.t, "gN": float(gN * up), "h": float(h), "rb": float(rb * up),
            "P": P, "rho": rho}


def lemma0_margin(N: int, cmax: int = 1 << 29, digits: int = 60) -> tuple:
    """The exhaustive evaluation in the proof of Lemma 0, for P' of N moduli.

    The proof states that, for every P' of eq. (p_list) and every
    e' = log2(cbar) with cbar an integer in [1, 2^29] (cbar <= 2^12 k, k <= 2^17),
        floor(P' - 0.5 (1 + u32) e') <= P' - 0.5 e' - 2^-21,
    with 2^-21 found empirically.  Returns (margin, cbar): the smallest
    P' - 0.5 e' - floor(P' - 0.5 (1 + u32) e') over all those cbar, and the
    cbar where it occurs.

    Over the cbar whose floor takes one value kf, the margin P' - 0.5 log2(cbar) - kf
    falls as cbar grows, so each kf contributes only its largest cbar: the largest
    integer with log2(cbar) <= 2 (P' - kf) / (1 + u32), clipped to cmax.  That
    keeps the evaluation exhaustive at about 15 candidates per N.
    """
    Pp = Fraction(float(constants(N).Pprime))
    one_u = 1 + U32
    best = None
    with localcontext() as ctx:
        ctx.prec = digits
        ln2 = Decimal(2).ln()

        def log2d(c: int) -> Decimal:
            return Decimal(c).ln() / ln2

        def dec(fr: Fraction) -> Decimal:
            return Decimal(fr.numerator) / Decimal(fr.denominator)

        def floor_F(c: int) -> int:
            # floor(P' - 0.5 (1 + u32) log2 c), exactly for powers of two
            if c & (c - 1) == 0:
                v = Pp - one_u * Fraction(c.bit_length() - 1, 2)
                return math.floor(v)
            v = dec(Pp) - dec(one_u) * log2d(c) / 2
            f = math.floor(v)
            assert abs(v - f) > Decimal(10) ** (10 - digits) and abs(v - f - 1) > Decimal(10) ** (10 - digits)
            return f

        def margin(c: int) -> Decimal:
            return dec(Pp) - log2d(c) / 2 - floor_F(c)

        k_lo = floor_F(cmax)
        k_hi = math.floor(Pp)
        for kf in range(k_lo, k_hi + 1):
            X = dec(2 * (Pp - kf) / one_u)                       # log2(cbar) <= X
            if X < 0:
                continue
            c = int((X * ln2).exp().to_integral_value(rounding="ROUND_FLOOR"))
            c = min(max(c, 1), cmax)
            while c < cmax and floor_F(c + 1) >= kf:              # guard against rounding in exp()
                c += 1
            while c > 1 and floor_F(c) < kf:
                c -= 1
            if floor_F(c) != kf:
                continue                                          # no integer cbar has this floor
            m = margin(c)
            if best is None or m < best[0]:
                best = (m, c)
    return best
