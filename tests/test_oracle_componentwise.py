"""Pins of the oracle's componentwise N rule (ozaki2.choose_N_componentwise), a
reading of Theorem 2: its bound holds entry by entry (eq. thm:err-1), so N can
be chosen to make the N-dependent part of that bound at most tau (|A||B|)_ij on
every entry.  The rule needs a lower bound of (|A||B|)_ij; it takes
L_ij = 2^-(mu'_i + nu'_j) (floor(2^mu' |A|) floor(|B| 2^nu'))_ij.

Pinned here with exact rationals (Python Fractions and integers):
* L_ij <= (|A||B|)_ij on every entry, subnormal and huge inputs included;
* at the chosen N the exact N-dependent part of eq. thm:err-1 is at most
  tau (|A||B|)_ij on every entry, and N - 1 misses the rule's criterion;
* the emulated product's error is at most tau (|A||B|)_ij plus the
  N-independent rest of eq. thm:err-1;
* a planted mistake (ceil instead of floor in L) breaks the first pin.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki2 as oz
from oracle.constants import U64, constants
from paper_2602_02549_b300.inputs import paper_pair, wide_exponent_matrix

from test_oracle_bounds import F, bars, exact_abs_sum, gN_exact, t_interval, sqrt_interval


def exact_absAB(A, B):
    m, k = A.shape
    n = B.shape[1]
    FA = [[abs(F(A[i, h])) for h in range(k)] for i in range(m)]
    FB = [[abs(F(B[h, j])) for j in range(n)] for h in range(k)]
    return [[sum(FA[i][h] * FB[h][j] for h in range(k)) for j in range(n)] for i in range(m)]


def lower_exact(A, B):
    """L_ij with Python integers, from alpha and beta taken from the entries' exponents."""
    alpha, beta, _, _, _ = bars(A, B)
    m, k = A.shape
    n = B.shape[1]
    mu = [5 - a if a is not None else 0 for a in alpha]
    nu = [5 - b if b is not None else 0 for b in beta]
    Ah = [[math.floor(abs(F(A[i, h])) * Fraction(2) ** mu[i]) for h in range(k)] for i in range(m)]
    Bh = [[math.floor(abs(F(B[h, j])) * Fraction(2) ** nu[j]) for j in range(n)] for h in range(k)]
    return [[Fraction(sum(Ah[i][h] * Bh[h][j] for h in range(k))) * Fraction(2) ** -(mu[i] + nu[j])
             for j in range(n)] for i in range(m)]


INPUTS = [("paper", 6, 5, 40, 0.5), ("paper", 5, 7, 60, 1.0), ("paper", 4, 4, 33, 2.0), ("wide", 5, 6, 20, 0.0)]


def make(kind, m, n, k, phi, seed):
    if kind == "paper":
        return paper_pair(m, n, k, phi, seed=seed)
    return (wide_exponent_matrix(m, k, -1070, 600, seed, zero_frac=0.2),
            wide_exponent_matrix(k, n, -900, 500, seed + 1, zero_frac=0.2))


@pytest.mark.parametrize("inp", INPUTS)
def test_lower_bound_is_exact_lower_bound(inp):
    A, B = make(*inp, seed=7)
    s = oz.scaling(A, B, 14)
    L = oz.componentwise_lower(A, B, s["mu_p"], s["nu_p"])
    Lx = lower_exact(A, B)
    AB = exact_absAB(A, B)
    m, n = L.shape
    for i in range(m):
        for j in range(n):
            assert F(L[i, j]) == Lx[i][j]          # ldexp of an exact integer sum
            assert Lx[i][j] <= AB[i][j]


def npart_interval(A, B, N, b, i, j, s):
    """[lo, hi] of the N-dependent part of eq. thm:err-1 at entry (i, j)."""
    k = A.shape[1]
    P = constants(N, b).P
    tl, th = t_interval(P)
    R = exact_abs_sum(A[i])
    K = exact_abs_sum(B[:, j])

    def p2(e, c):
        if e == oz.INT32_MIN or c == 0:
            return Fraction(0), Fraction(0)
        lo, hi = sqrt_interval(Fraction(int(c)))
        return lo * Fraction(2) ** int(e), hi * Fraction(2) ** int(e)
    a2 = p2(s["alpha"][i], s["cmax_row"][i])
    b2 = p2(s["beta"][j], s["cmax_col"][j])
    c = k + gN_exact(N, b)
    lo = tl * R * b2[0] + tl * a2[0] * K + c * tl * tl * a2[0] * b2[0]
    hi = th * R * b2[1] + th * a2[1] * K + c * th * th * a2[1] * b2[1]
    return lo, hi


@pytest.mark.parametrize("tau", [1e-8, 1e-12, 1e-15])
@pytest.mark.parametrize("inp", INPUTS[:3])
def test_chosen_N_meets_target_on_every_entry(inp, tau):
    A, B = make(*inp, seed=11)
    s = oz.scaling(A, B, 14)
    N, info = oz.choose_N_componentwise(A, B, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], tau, 49)
    if N > 2:
        assert info["ratios"][N - 1] > tau
    if info["ratios"][N] > tau:                # nmax: no N meets the target
        assert N == 49
        return
    AB = exact_absAB(A, B)
    m, n = len(AB), len(AB[0])
    for i in range(m):
        for j in range(n):
            _, hi = npart_interval(A, B, N, 64, i, j, s)
            assert hi <= Fraction(tau) * AB[i][j]
    # the emulated product: error within tau (|A||B|)_ij plus the N-independent rest of err-1
    r = oz.os_ii(A, B, N, 64)
    err = np.abs(oz.exact_residual(A, B, r["C"]))
    e1, _ = oz.bounds(A, B, r)
    for i in range(m):
        for j in range(n):
            lo, _ = npart_interval(A, B, N, 64, i, j, s)
            rest = F(e1[i, j]) - lo                     # an upper bound of the N-independent part
            assert F(err[i, j]) <= Fraction(tau) * AB[i][j] + rest


def test_exponent_spread_forces_nmax():
    # phi = 4: many entries quantise to zero after the row / column scaling, so
    # some L_ij vanish while their bound terms do not; the rule can then only
    # answer nmax (the normwise rule still picks a small N)
    A, B = paper_pair(64, 64, 512, 4.0, seed=3)
    s = oz.scaling(A, B, 14)
    N, info = oz.choose_N_componentwise(A, B, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], 1e-15, 30)
    assert N == 30 and not np.isfinite(info["xmax"])
    Nn, _ = oz.choose_N(A, B, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], 1e-15, 30)
    assert Nn < 30


def test_planted_ceil_lower_bound_is_caught(monkeypatch):
    # ceil instead of floor: no longer a lower bound of (|A||B|)_ij
    orig = oz.floor_scaled_abs

    def ceil_scaled(X, shift, axis):
        Xa = np.abs(np.asarray(X, np.float64))
        sh = np.asarray(shift, np.int64)
        return np.ceil(np.ldexp(Xa, sh[:, None] if axis == 1 else sh[None, :])).astype(np.int8)
    monkeypatch.setattr(oz, "floor_scaled_abs", ceil_scaled)
    A, B = make(*INPUTS[0], seed=7)
    s = oz.scaling(A, B, 14)
    L = oz.componentwise_lower(A, B, s["mu_p"], s["nu_p"])
    AB = exact_absAB(A, B)
    assert any(F(L[i, j]) > AB[i][j] for i in range(L.shape[0]) for j in range(L.shape[1]))
    monkeypatch.setattr(oz, "floor_scaled_abs", orig)
