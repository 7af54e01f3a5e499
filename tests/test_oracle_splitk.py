"""Pins of the oracle's split-K extension (k > 2^17, outside the paper's
assumption k <= 2^17 of Section 3): consecutive K ranges, one OS_II each,
results added in range order.

* the ranges partition [0, k) with at most 2^17 each (and the library's
  oz2_k_ranges, computed independently in C, gives the same split);
* integer inputs with A' = A, B' = B (mu = nu = 0 injected) and N = 5, where
  every range is exact (s_l2 = P2 = 0), sum to the exact product bit for bit;
* the summed bound (the ranges' Theorem 2 bounds from their exponents plus one
  rounding per addition) holds against the exact product, and fails when a
  range is left out (a planted mistake, on the CPU).
"""
import numpy as np
import pytest

from oracle.constants import K_MAX
from paper_2602_02549_b300.inputs import integer_matrix, paper_pair


@pytest.mark.parametrize("k", [1, 63, K_MAX - 1, K_MAX, K_MAX + 1, 2 * K_MAX, 2 * K_MAX + 1,
                               3 * K_MAX - 5, 1_000_003, 2**31 - 1])
def test_ranges_partition(oracle, k):
    r = oracle.splitk_ranges(k)
    assert r[0][0] == 0 and r[-1][1] == k
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    assert all(0 < k1 - k0 <= K_MAX for k0, k1 in r)
    assert len(r) <= -(-k // K_MAX)
    if k <= K_MAX:
        assert r == [(0, k)]
    else:
        assert all((k1 - k0) % 64 == 0 for k0, k1 in r[:-1])


def test_ranges_match_library(oracle):
    from paper_2602_02549_b300 import binding as B
    rng = np.random.default_rng(3)
    ks = [1, 2, K_MAX - 1, K_MAX, K_MAX + 1, 2 * K_MAX, 2**31 - 1] + [int(x) for x in rng.integers(1, 2**31 - 1, 200)]
    for k in ks:
        r = oracle.splitk_ranges(k)
        count, kc = B.k_ranges(k)
        assert count == len(r) and kc == r[0][1] - r[0][0], k


def test_one_range_is_os_ii(oracle):
    A, Bm = paper_pair(20, 12, 700, 1.0, seed=2)
    a = oracle.os_ii(A, Bm, 9)
    b = oracle.os_ii_splitk(A, Bm, 9)
    assert np.array_equal(a["C"].view(np.int64), b["C"].view(np.int64))


def test_integer_inputs_exact(oracle):
    # every range exact at N = 5 (A' = A, B' = B, |A'B'| <= 5 * 5 * 2^17 < P/2),
    # and the FP64 sums of integers below 2^53 are exact
    k = K_MAX + 4099
    A = integer_matrix(3, k, -5, 5, seed=11)
    Bm = integer_matrix(k, 2, -5, 5, seed=12)
    ranges = oracle.splitk_ranges(k)
    z3, z2 = [np.zeros(3, np.int32)] * len(ranges), [np.zeros(2, np.int32)] * len(ranges)
    r = oracle.os_ii_splitk(A, Bm, 5, mu_in=z3, nu_in=z2)
    exact = A.astype(np.int64) @ Bm.astype(np.int64)
    assert len(ranges) == 2
    assert np.array_equal(r["C"], exact.astype(np.float64))


@pytest.mark.parametrize("b", [64, 32])
def test_summed_bound(oracle, b):
    k = K_MAX + 3000
    dt = np.float64 if b == 64 else np.float32
    A, Bm = paper_pair(4, 3, k, 1.0, seed=5, dtype=dt)
    A, Bm = A.astype(np.float64), Bm.astype(np.float64)
    N = 10 if b == 64 else 6
    r = oracle.os_ii_splitk(A, Bm, N, b)
    C = r["C"].astype(np.float64)
    eb = oracle.bound_splitk(A, Bm, r, b)
    err = np.abs(oracle.exact_residual(A, Bm, C))
    assert (err <= eb).all()
    # planted mistake: the second range left out
    bad = r["parts"][0]["C"].astype(np.float64)
    assert (np.abs(oracle.exact_residual(A, Bm, bad)) > eb).any()
