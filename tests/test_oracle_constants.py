"""Pins of the oracle's constant tables against exact integer facts.

Each check uses a formulation different from the one in oracle/constants.py
(integer bit masks instead of rational floors, Python's % instead of pow(),
math.log2 on big integers instead of Decimal), so a transcription or rounding
mistake in the tables fails here.
"""
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle.constants import MODULI, constants, U32, U64

HERE = os.path.dirname(os.path.abspath(__file__))
FACTS = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))
ALL_N = list(range(2, 50))


def test_moduli_match_paper_list():
    # Section 3.1, eq. (p_list)
    assert list(MODULI) == FACTS["moduli"]["values"]
    assert len(MODULI) == FACTS["n_max"]["value"]
    assert all(2 <= p <= 256 for p in MODULI)
    for i, a in enumerate(MODULI):
        for b in MODULI[i + 1:]:
            assert math.gcd(a, b) == 1          # Theorem 1: pairwise coprime


@pytest.mark.parametrize("N", ALL_N)
def test_q_is_inverse(N):
    # Theorem 1 and Step 1: (P/p_l) q_l = 1 mod p_l, q_l < p_l
    C = constants(N)
    for pl, ql in zip(C.p, C.q):
        assert 1 <= ql < pl
        assert ((C.P // pl) % pl) * ql % pl == 1


@pytest.mark.parametrize("N", [2, 3, 5, 8, 14, 20, 33, 49])
def test_crt_round_trip(N):
    # Theorem 1: x = mod(sum P/p_l q_l y_l, P) when 2|x| < P
    C = constants(N)
    rng = random.Random(N)
    samples = [0, 1, -1, (C.P - 1) // 2, -((C.P - 1) // 2)]
    samples += [rng.randrange(-(C.P // 2) + 1, C.P // 2) for _ in range(200)]
    for x in samples:
        ys = [x % pl for pl in C.p]
        S = sum(xl * y for xl, y in zip(C.x, ys)) % C.P
        if 2 * S >= C.P:
            S -= C.P
        assert S == x


@pytest.mark.parametrize("N", ALL_N)
def test_s1_s2_dgemm(N):
    # Section 3.1: s_l1 keeps the upper beta_l bits of P/p_l q_l; s_l2 = double(rest)
    C = constants(N, 64)
    rho = sum(p // 2 for p in C.p)
    assert C.rho == rho
    clog_rho = (rho - 1).bit_length()
    r = max(C.x)
    for xl, s1, s2 in zip(C.x, C.s1, C.s2):
        beta = 53 - clog_rho + (xl.bit_length() - 1) - (r.bit_length() - 1)
        drop = xl.bit_length() - beta               # low bits removed
        kept = (xl >> drop) << drop if drop > 0 else xl
        assert Fraction(s1) == kept
        rest = xl - kept
        assert 0 <= rest < 2 ** (1 + clog_rho) * U64 * C.P   # proof of Lemma 2
        assert s2 == float(rest)                    # correctly rounded
    if N <= 5:
        assert all(s == 0.0 for s in C.s2)


@pytest.mark.parametrize("N", ALL_N)
def test_s1_sgemm(N):
    C = constants(N, 32)
    for xl, s1, s2 in zip(C.x, C.s1, C.s2):
        assert s2 == 0.0
        assert abs(Fraction(s1) - xl) <= Fraction(xl) * U64     # double(P/p_l q_l)
    assert C.P2 == 0.0


@pytest.mark.parametrize("N", ALL_N)
def test_P1_P2_Pinv(N):
    C = constants(N, 64)
    P = C.P
    # P1 = double(P): nearest double
    e = P.bit_length() - 53
    ulp = 2 ** max(e, 0)
    assert abs(int(C.P1) - P) * 2 <= ulp
    # eq. (errP): |P1 + P2 - P| <= u^2 P / 2
    assert abs(Fraction(C.P1) + Fraction(C.P2) - P) <= U64 ** 2 * P / 2
    if P < 2 ** 53:
        assert C.P2 == 0.0 and int(C.P1) == P
    # P_inv = double(1/P)
    assert abs(Fraction(C.Pinv) - Fraction(1, P)) <= U64 * Fraction(1, P)


@pytest.mark.parametrize("N", ALL_N)
def test_Pprime(N):
    # Algorithm 2: P' = single_down(log2(P-1)/2 - 0.5); Section 3.2: P' < 200
    C = constants(N)
    v = math.log2(C.P - 1) / 2 - 0.5
    f = float(C.Pprime)
    nxt = float(np.nextafter(C.Pprime, np.float32(np.inf)))
    slack = 1e-12 * v
    assert f <= v + slack and v < nxt + slack
    assert f < FACTS["pprime_max"]["value"]
    assert isinstance(C.Pprime, np.float32)


def test_c_constant():
    # Algorithm 2: c = single_down(-0.5/(1-4 u32)); -0.5/(1-2^-22) = -0.5 - 2^-23 - ...,
    # FP32 spacing in [0.5, 1) is 2^-24, so the largest float below is -(0.5 + 3*2^-24).
    C = constants(14)
    assert C.c == np.float32(-(0.5 + 3 * 2.0 ** -24))
    assert Fraction(float(C.c)) <= Fraction(-1, 2) / (1 - 4 * U32)


def test_paper_unit_roundoffs():
    assert float(U32) == FACTS["u32"]["value"]
    assert float(U64) == FACTS["u64"]["value"]


@pytest.mark.parametrize("N", [2, 14, 49])
def test_p256_is_first(N):
    # eq. (p_list): 256 first; INT8 wrap argument of Section 3.1
    assert constants(N).p[0] == 256


# ---------------------------------------------------------------- Lemma 0's constant
# The proof of Lemma 0 rests on an exhaustive evaluation: for every P' of
# eq. (p_list) and every e' = log2(cbar), cbar an integer in [1, 2^29],
#   floor(P' - 0.5 (1 + u32) e') <= P' - 0.5 e' - 2^-21,
# with 2^-21 found empirically, i.e. the smallest margin lies in [2^-21, 2^-20).
def test_lemma0_exhaustive_constant():
    from decimal import Decimal
    from oracle.constants import lemma0_margin
    worst = min(lemma0_margin(N)[0] for N in range(2, 50))
    assert Decimal(2) ** -21 <= worst < Decimal(2) ** -20


@pytest.mark.parametrize("N", [2, 9, 17, 32, 49])
def test_lemma0_margin_brute_force(N):
    """The oracle's reduction to one candidate per floor value against every
    cbar up to 2^16, evaluated directly (float64 log2, and mpmath at 50 digits
    wherever float64 cannot decide the floor)."""
    import mpmath
    from oracle.constants import lemma0_margin
    cmax = 1 << 16
    Pp = float(constants(N).Pprime)
    c = np.arange(1, cmax + 1, dtype=np.float64)
    e = np.log2(c)
    F = Pp - 0.5 * (1 + 2.0 ** -24) * e
    fl = np.floor(F)
    m = Pp - 0.5 * e - fl
    close = (F - fl < 1e-9) | (fl + 1 - F < 1e-9)
    mpmath.mp.dps = 50
    for idx in np.nonzero(close)[0]:
        cc = int(idx) + 1
        ee = mpmath.log(cc, 2)
        Fx = mpmath.mpf(Pp) - mpmath.mpf(1 + 2.0 ** -24) / 2 * ee
        m[idx] = float(mpmath.mpf(Pp) - ee / 2 - mpmath.floor(Fx))
    brute = m.min()
    got, cg = lemma0_margin(N, cmax=cmax)
    assert abs(float(got) - brute) < 1e-12
    assert abs(m[cg - 1] - brute) < 1e-12
