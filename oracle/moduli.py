"""Per-N moduli tables: for each N, the N pairwise coprime integers <= 256 with
the largest product P (Section 3.1 fixes one list, eq. (p_list), whose first N
entries serve every N, and remarks that tables chosen per N could refine the
method).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only the test suite may
import this module.

The search keeps the structure the implementation relies on: the first modulus
is 256 = 2^8 (the largest power of two; its residues are low bytes), and the
other N - 1 are odd.  Choosing them is a 0/1 program over the odd candidates
c in [3, 255]: maximise sum log(c) with exactly N - 1 chosen and, for every odd
prime q <= 255, at most one chosen multiple of q (pairwise coprime).  scipy's
MILP (HiGHS) solves it; best_products() checks the answer with exact integers
(coprimality, the product) and, for small N, against an exhaustive
branch-and-bound over integer products (exhaustive_best).

    python -m oracle.moduli [--compare]

prints the tables and, with --compare, how the bound rule's N changes with
them (compare_rule).
"""
from __future__ import annotations

import math
import sys
from functools import lru_cache

import numpy as np

from .constants import MODULI, N_MAX, N_MIN, U64

ODD = tuple(range(3, 256, 2))


def odd_primes(limit: int = 255) -> list[int]:
    return [q for q in range(3, limit + 1, 2) if all(q % d for d in range(3, math.isqrt(q) + 1, 2))]


def pairwise_coprime(ps) -> bool:
    ps = list(ps)
    return all(math.gcd(a, b) == 1 for i, a in enumerate(ps) for b in ps[i + 1:])


@lru_cache(maxsize=None)
def optimal_moduli(N: int) -> tuple:
    """(256, c_2, ..., c_N): the odd c pairwise coprime with the largest product,
    in descending order (the 0/1 program above)."""
    from scipy.optimize import Bounds, LinearConstraint, milp
    if not (N_MIN <= N <= N_MAX):
        raise ValueError("N must be in [2, 49]")
    cand = np.array(ODD)
    primes = odd_primes()
    A = np.zeros((len(primes) + 1, len(cand)))
    for r, q in enumerate(primes):
        A[r] = (cand % q == 0)
    A[-1] = 1.0
    lo = np.zeros(len(primes) + 1)
    hi = np.ones(len(primes) + 1)
    lo[-1] = hi[-1] = N - 1
    res = milp(c=-np.log(cand.astype(np.float64)), constraints=LinearConstraint(A, lo, hi),
               integrality=np.ones(len(cand)), bounds=Bounds(0, 1),
               options={"mip_rel_gap": 0.0, "presolve": True})
    if not res.success:
        raise RuntimeError(f"MILP failed for N={N}: {res.message}")
    chosen = sorted((int(c) for c, x in zip(cand, res.x) if x > 0.5), reverse=True)
    out = (256,) + tuple(chosen)
    assert len(out) == N and pairwise_coprime(out)
    return out


def exhaustive_best(N: int) -> int:
    """The largest product of 256 and N - 1 pairwise coprime odd integers <= 255,
    by depth-first search over descending candidates with exact integer products,
    pruned by the bound product * (largest remaining candidate)^(slots left)."""
    best = [0]

    def dfs(start: int, slots: int, prod: int, used: tuple):
        if slots == 0:
            best[0] = max(best[0], prod)
            return
        for i in range(start, len(ODD_DESC)):
            c = ODD_DESC[i]
            if prod * c ** slots <= best[0]:
                return                       # candidates only get smaller from here
            if any(math.gcd(c, u) != 1 for u in used):
                continue
            dfs(i + 1, slots - 1, prod * c, used + (c,))
    dfs(0, N - 1, 256, ())
    return best[0]


ODD_DESC = tuple(sorted(ODD, reverse=True))


def product(ps) -> int:
    return math.prod(ps)


def rule_terms(ps, N: int) -> dict:
    """t = 1/sqrt(2^5 (P-1)) (rounded up) and g_N, the P-proportional part of
    R_64 (Lemma 4), for the moduli ps (b = 64)."""
    from fractions import Fraction
    P = product(ps)
    rho = sum(p // 2 for p in ps)
    t = 1.0 / math.sqrt(32.0 * float(P - 1)) * (1.0 + 2.0 ** -50)
    gN = (1 + 3 * U64) * Fraction(2) ** (1 + (rho - 1).bit_length()) * (N + 2) * U64 ** 2 * rho * P
    return {"t": t, "gN": float(gN * (1 + Fraction(1, 1 << 40))), "P": P, "rho": rho}


def rule_N(maxima: dict, k: int, tau: float, nmax: int, tables) -> int:
    """The normwise bound rule (ozaki2.choose_N_from_maxima) with the moduli
    tables(N) for each N."""
    for N in range(N_MIN, nmax + 1):
        bt = rule_terms(tables(N), N)
        t = bt["t"]
        T = t * (maxima["maxR"] * maxima["max2b"] + maxima["max2a"] * maxima["maxK"]) + \
            (k + bt["gN"]) * t * t * maxima["max2a"] * maxima["max2b"]
        if T <= tau * maxima["L"]:
            return N
    return nmax


def compare_rule(problems, tau: float = 1e-15, nmax: int = 49) -> list:
    """For each (A, B): the bound rule's N with the paper's list and with the
    per-N optimal tables (same scaling, same maxima)."""
    from . import ozaki2 as oz
    out = []
    for A, B in problems:
        s = oz.scaling(A, B, 14)
        _, info = oz.choose_N(A, B, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], tau, nmax)
        mx = {k: info[k] for k in ("maxR", "maxK", "max2a", "max2b", "L")}
        k = A.shape[1]
        out.append((rule_N(mx, k, tau, nmax, lambda N: MODULI[:N]), rule_N(mx, k, tau, nmax, optimal_moduli)))
    return out


def main(argv) -> None:
    print("N  log2 P (paper)  log2 P (per-N)  gain (bits)  moduli")
    for N in range(N_MIN, N_MAX + 1):
        a, b = product(MODULI[:N]), product(optimal_moduli(N))
        print(f"{N:2d}  {math.log2(a):13.3f}  {math.log2(b):14.3f}  {math.log2(b) - math.log2(a):11.3f}  "
              f"{optimal_moduli(N)}")
    if "--compare" in argv:
        from paper_2602_02549_b300.inputs import batched_specs, paper_pair
        probs = []
        for i, (m, n, k, phi) in enumerate(batched_specs(64, 0)):
            if m * n * k <= 2 ** 31:              # the oracle's Cbar within seconds
                probs.append(paper_pair(m, n, k, phi, seed=2 * i))
        for phi in (0.5, 1.0, 2.0, 4.0):
            for size in (512, 1024, 2048):
                probs.append(paper_pair(size, size, size, phi, seed=int(10 * phi) + size))
        res = compare_rule(probs)
        changed = [(i, a, b) for i, (a, b) in enumerate(res) if a != b]
        print(f"tau = 1e-15: {len(res)} problems, N changed for {len(changed)}: {changed}")


if __name__ == "__main__":
    main(sys.argv[1:])
