"""Pins of the oracle's bound evaluators against the paper's bounds evaluated
independently in exact rational arithmetic.

* bounds():               eq. thm:err-1 and eq. thm:err-2 of Theorem 2;
* bound_from_exponents(): Lemma 1's truncation bound with the exponents used
                          (|Delta_A|, |Delta_B| < 1 in its proof) plus Lemma 4's R_b;
* bound_splitk():         that bound summed over the K ranges, plus one rounding
                          of the running sum per addition;
* mu_band():              Algorithm 2's mu line over every FP32 e that
                          assumption (1) of Section 1.2 admits.

Everything here is recomputed from A and B with Python integers and Fractions:
alpha, beta from the exponents of the entries, Abar, Bbar and Cbar = Abar Bbar
as integers, |A'B'| from A' = trunc(2^mu A) taken exactly, the 1-norms as exact
sums.  The irrational factors (t = 1/sqrt(2^5 (P-1)) and sqrt(max cbar)) are
enclosed in rational intervals 2^-100 wide, so the exact bound lies in
[lo, hi].  The oracle's FP64 value must be >= hi (a valid upper bound) and
<= lo (1 + 2^-36): no looser than its own safety factors (a few factors of
1 + 2^-40 and FP64 roundings, about 2^-38 in all).

Planted mistakes (monkeypatched into the oracle module, on the CPU) show that a
plausible error in any of these evaluators fails at least one pin.
"""
import math
from decimal import Decimal, localcontext
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki2 as oz
from oracle.constants import U32, U64, constants
from paper_2602_02549_b300.inputs import paper_pair

SLACK = Fraction(1) + Fraction(1, 1 << 36)
PREC = 100   # bits of the interval enclosures


# --------------------------------------------------------------------------- #
# Exact helpers (no oracle code)
# --------------------------------------------------------------------------- #
def F(x) -> Fraction:
    n, d = float(x).as_integer_ratio()
    return Fraction(n, d)


def floor_log2_abs(x: float) -> int:
    """floor(log2 |x|) of a nonzero double, exactly (frexp gives |x| = f 2^e, f in [1/2, 1))."""
    return math.frexp(abs(float(x)))[1] - 1


def sqrt_interval(x: Fraction) -> tuple[Fraction, Fraction]:
    """lo <= sqrt(x) <= hi for a nonnegative rational, hi - lo ~ 2^-PREC sqrt(x)."""
    if x == 0:
        return Fraction(0), Fraction(0)
    num, den = x.numerator, x.denominator
    # sqrt(num/den) = sqrt(num den) / den
    s = max(0, PREC + 4 - (num * den).bit_length() // 2)
    r = math.isqrt(num * den << (2 * s))
    return Fraction(r, den << s), Fraction(r + 1, den << s)


def t_interval(P: int) -> tuple[Fraction, Fraction]:
    """t = 1/sqrt(2^5 (P-1)) (Theorem 2) enclosed."""
    lo, hi = sqrt_interval(Fraction(32 * (P - 1)))
    return 1 / hi, 1 / lo


def gN_exact(N: int, b: int) -> Fraction:
    """The P-proportional part of R_b (Lemma 4, Theorem 2)."""
    C = constants(N, b)
    rho, P = C.rho, C.P
    if b == 64:
        return (1 + 3 * U64) * Fraction(2) ** (1 + (rho - 1).bit_length()) * (N + 2) * U64 ** 2 * rho * P
    return (1 + U32) * (N + 2) * U64 * rho * P


def h_exact(b: int) -> Fraction:
    """The coefficient of |A'B'| in R_b (Lemma 4)."""
    return 3 * U64 if b == 64 else U32


def rb_exact(N: int, b: int) -> Fraction:
    """r_b of eq. thm:err-2 (|A'B'| replaced by P/2 via Lemma 0)."""
    P = constants(N, b).P
    return gN_exact(N, b) + (Fraction(3, 2) * U64 * P if b == 64 else Fraction(1, 2) * U32 * P)


def exact_abs_sum(xs) -> Fraction:
    return sum((abs(F(v)) for v in xs), Fraction(0))


def bars(A: np.ndarray, B: np.ndarray):
    """alpha, beta, Abar, Bbar (Algorithm 2) and Cbar = Abar Bbar as Python ints."""
    m, k = A.shape
    n = B.shape[1]
    alpha = [max((floor_log2_abs(v) for v in A[i] if v != 0), default=None) for i in range(m)]
    beta = [max((floor_log2_abs(v) for v in B[:, j] if v != 0), default=None) for j in range(n)]
    Abar = [[math.ceil(abs(F(A[i, h])) * Fraction(2) ** (5 - alpha[i])) if alpha[i] is not None else 0
             for h in range(k)] for i in range(m)]
    Bbar = [[math.ceil(abs(F(B[h, j])) * Fraction(2) ** (5 - beta[j])) if beta[j] is not None else 0
             for j in range(n)] for h in range(k)]
    Cbar = [[sum(Abar[i][h] * Bbar[h][j] for h in range(k)) for j in range(n)] for i in range(m)]
    return alpha, beta, Abar, Bbar, Cbar


def trunc_scaled(x: float, s: int) -> int:
    """trunc(2^s x), exactly."""
    v = F(x) * Fraction(2) ** int(s)
    return math.trunc(v)


def exact_ApBp(A, B, mu, nu):
    m, k = A.shape
    n = B.shape[1]
    Ap = [[trunc_scaled(A[i, h], mu[i]) for h in range(k)] for i in range(m)]
    Bp = [[trunc_scaled(B[h, j], nu[j]) for j in range(n)] for h in range(k)]
    return [[sum(Ap[i][h] * Bp[h][j] for h in range(k)) for j in range(n)] for i in range(m)]


def theorem2_intervals(A, B, N, b, mu, nu):
    """[lo, hi] enclosures of eq. thm:err-1 and eq. thm:err-2 on every entry."""
    m, k = A.shape
    n = B.shape[1]
    P = constants(N, b).P
    alpha, beta, _, _, Cbar = bars(A, B)
    cmax_row = [max(r) for r in Cbar]
    cmax_col = [max(Cbar[i][j] for i in range(m)) for j in range(n)]
    tl, th = t_interval(P)
    ApBp = exact_ApBp(A, B, mu, nu)
    gN, h, rb = gN_exact(N, b), h_exact(b), rb_exact(N, b)
    R = [exact_abs_sum(A[i]) for i in range(m)]
    K = [exact_abs_sum(B[:, j]) for j in range(n)]

    def p2(e, c):                      # 2^alpha' = 2^alpha sqrt(max cbar), enclosed
        if e is None or c == 0:
            return Fraction(0), Fraction(0)
        lo, hi = sqrt_interval(Fraction(c))
        return lo * Fraction(2) ** e, hi * Fraction(2) ** e

    a2 = [p2(alpha[i], cmax_row[i]) for i in range(m)]
    b2 = [p2(beta[j], cmax_col[j]) for j in range(n)]
    out1 = [[None] * n for _ in range(m)]
    out2 = [[None] * n for _ in range(m)]
    for i in range(m):
        for j in range(n):
            def ev(t, A2, B2, third):
                return t * R[i] * B2 + t * A2 * K[j] + third * t * t * A2 * B2
            c1 = k + gN + h * abs(ApBp[i][j])
            c2 = k + rb
            out1[i][j] = (ev(tl, a2[i][0], b2[j][0], c1), ev(th, a2[i][1], b2[j][1], c1))
            out2[i][j] = (ev(tl, a2[i][0], b2[j][0], c2), ev(th, a2[i][1], b2[j][1], c2))
    return out1, out2


def within(value: float, lohi) -> bool:
    lo, hi = lohi
    v = F(value)
    return hi <= v <= lo * SLACK


# --------------------------------------------------------------------------- #
# Cases: small shapes, the paper's generator, N spanning the regimes where the
# truncation terms (small N) and the FP64 / FP32 output rounding (large N)
# dominate the bound
# --------------------------------------------------------------------------- #
CASES = [(3, 4, 5, 0.5), (4, 3, 7, 2.0), (2, 5, 6, 4.0)]
NS = [2, 3, 5, 8, 14, 20, 49]


def case_inputs(case, N, b):
    m, n, k, phi = case
    dt = np.float64 if b == 64 else np.float32
    A, B = paper_pair(m, n, k, phi, seed=3 * N + m + b, dtype=dt)
    return A.astype(np.float64), B.astype(np.float64)


def check_theorem2(A, B, N, b) -> bool:
    r = oz.os_ii(A, B, N, b)
    e1, e2 = oz.bounds(A, B, r)
    x1, x2 = theorem2_intervals(A, B, N, b, r["mu"], r["nu"])
    m, n = e1.shape
    return all(within(e1[i, j], x1[i][j]) and within(e2[i, j], x2[i][j]) for i in range(m) for j in range(n))


@pytest.mark.parametrize("b", [64, 32])
@pytest.mark.parametrize("N", NS)
@pytest.mark.parametrize("case", CASES)
def test_theorem2_bounds_exact(case, N, b):
    A, B = case_inputs(case, N, b)
    assert check_theorem2(A, B, N, b)


def test_theorem2_zero_rows_columns():
    # rows / columns excluded by Theorem 2's assumption carry the terms they have:
    # a zero row of A gives R_i = 0 and 2^alpha'_i = 0, so only t 2^... vanish
    A, B = paper_pair(4, 4, 6, 1.0, seed=9)
    A[1, :] = 0.0
    B[:, 2] = 0.0
    for N in (2, 14):
        assert check_theorem2(A, B, N, 64)


def exponent_bound_exact(A, B, N, b, mu, nu):
    m, k = A.shape
    n = B.shape[1]
    ApBp = exact_ApBp(A, B, mu, nu)
    gN, h = gN_exact(N, b), h_exact(b)
    R = [exact_abs_sum(A[i]) for i in range(m)]
    K = [exact_abs_sum(B[:, j]) for j in range(n)]
    two = Fraction(2)
    return [[R[i] * two ** -int(nu[j]) + two ** -int(mu[i]) * K[j]
             + (k + gN + h * abs(ApBp[i][j])) * two ** -(int(mu[i]) + int(nu[j]))
             for j in range(n)] for i in range(m)]


def check_exponent_bound(A, B, N, b, mu=None, nu=None) -> bool:
    r = oz.os_ii(A, B, N, b, mu_in=mu, nu_in=nu)
    got = oz.bound_from_exponents(A, B, r["mu"], r["nu"], r["Ap"], r["Bp"], N, b)
    x = exponent_bound_exact(A, B, N, b, r["mu"], r["nu"])
    m, n = got.shape
    return all(within(got[i, j], (x[i][j], x[i][j])) for i in range(m) for j in range(n))


@pytest.mark.parametrize("b", [64, 32])
@pytest.mark.parametrize("N", NS)
def test_exponent_bound_exact(N, b):
    for case in CASES:
        A, B = case_inputs(case, N, b)
        assert check_exponent_bound(A, B, N, b)


def test_exponent_bound_injected_exponents():
    # the bound holds for any exponents that keep Lemma 0; here mu - 1, nu - 2
    A, B = paper_pair(3, 4, 8, 1.0, seed=4)
    s = oz.scaling(A, B, 14)
    assert check_exponent_bound(A, B, 14, 64, s["mu"] - 1, s["nu"] - 2)


# --------------------------------------------------------------------------- #
# Split-K: the sum of the ranges' exponent bounds plus one rounding per addition
# --------------------------------------------------------------------------- #
def exact_sum_abs_fast(xs) -> Fraction:
    """sum |x| of many doubles, exactly (integer numerators on the 2^-1074 grid)."""
    acc = 0
    for v in np.abs(np.asarray(xs, np.float64)).tolist():
        n, d = v.as_integer_ratio()
        acc += n << (1074 - (d.bit_length() - 1))
    return Fraction(acc, 1 << 1074)


def exact_dot_int(xs, ys) -> int:
    return sum(int(a) * int(b) for a, b in zip(xs, ys))


def splitk_bound_exact(A, B, res, b):
    u = U64 if b == 64 else U32
    eta = Fraction(1, 1 << 1075) if b == 64 else Fraction(1, 1 << 150)
    m, n = A.shape[0], B.shape[1]
    total = [[Fraction(0)] * n for _ in range(m)]
    two = Fraction(2)
    for s, ((k0, k1), r) in enumerate(zip(res["ranges"], res["parts"])):
        N = r["N"]
        gN, h = gN_exact(N, b), h_exact(b)
        R = [exact_sum_abs_fast(A[i, k0:k1]) for i in range(m)]
        K = [exact_sum_abs_fast(B[k0:k1, j]) for j in range(n)]
        Ap, Bp = r["Ap"], r["Bp"]             # integer-valued doubles: int() is exact
        for i in range(m):
            for j in range(n):
                ab = exact_dot_int(Ap[i], Bp[:, j])
                mu, nu = int(r["mu"][i]), int(r["nu"][j])
                total[i][j] += (R[i] * two ** -nu + two ** -mu * K[j]
                                + ((k1 - k0) + gN + h * abs(ab)) * two ** -(mu + nu) + eta)
                if s > 0:
                    total[i][j] += u * abs(F(res["partial"][s][i, j])) + eta
    return total


def check_splitk(A, B, res, b) -> bool:
    got = oz.bound_splitk(A, B, res, b)
    x = splitk_bound_exact(A, B, res, b)
    m, n = got.shape
    return all(within(got[i, j], (x[i][j], x[i][j])) for i in range(m) for j in range(n))


@pytest.fixture(scope="module")
def splitk_case():
    k = (1 << 17) + 2000
    A, B = paper_pair(3, 2, k, 1.0, seed=17)
    # N = 20: the output rounding, not the truncation, dominates each range's
    # bound, so the rounding of the additions is visible in the sum
    res = oz.os_ii_splitk(A, B, 20, 64)
    assert len(res["ranges"]) == 2
    return A, B, res


def test_splitk_bound_exact(splitk_case):
    A, B, res = splitk_case
    assert check_splitk(A, B, res, 64)


# --------------------------------------------------------------------------- #
# mu band: every FP32 e admitted by assumption (1), mu = mu' + floor(c e + P')
# --------------------------------------------------------------------------- #
def log2_dec(d: int) -> Decimal:
    with localcontext() as ctx:
        ctx.prec = 70
        return Decimal(d).ln() / Decimal(2).ln()


def admissible_e(d: int) -> list:
    """Every FP32 e with |e - log2 d| <= 4 u32 log2 d (assumption (1)), exactly."""
    if d & (d - 1) == 0:                         # log2 d is an integer: exact comparisons
        lg = Fraction(d.bit_length() - 1)
        tol = 4 * U32 * lg
        ok = lambda e: abs(F(e) - lg) <= tol    # noqa: E731
        start = np.float32(float(lg))
    else:
        with localcontext() as ctx:
            ctx.prec = 70
            lg = log2_dec(d)
            tol = Decimal(4) / Decimal(1 << 24) * lg

            def ok(e):
                n, q = float(e).as_integer_ratio()
                return abs(Decimal(n) / Decimal(q) - lg) <= tol
        start = np.float32(float(lg))
    assert ok(start)
    out = [start]
    e = start
    while True:
        e = np.nextafter(e, np.float32(-np.inf))
        if not ok(e):
            break
        out.append(e)
    e = start
    while True:
        e = np.nextafter(e, np.float32(np.inf))
        if not ok(e):
            break
        out.append(e)
    return out


def band_exact(d: int, N: int, b: int) -> tuple[int, int]:
    C = constants(N, b)
    vals = [math.floor(F(C.c) * F(e) + F(C.Pprime)) for e in admissible_e(d)]
    return min(vals), max(vals)


def near_threshold_ds(N: int, b: int, lo_rel: float, hi_rel: float, count: int = 6) -> list:
    """Integers d < 2^24 whose log2 d lies between lo_rel and hi_rel (in units of
    u32 log2 d) above a value of e where floor(c e + P') steps."""
    C = constants(N, b)
    c, Pp = float(C.c), float(C.Pprime)
    out = []
    for j in range(math.floor(Pp) - 12, math.floor(Pp) + 1):
        eb = (j - Pp) / c                        # c e + P' = j
        if not (2.0 < eb < 23.5):
            continue
        for rel in np.linspace(lo_rel, hi_rel, 5):
            d = int(round(2.0 ** (eb * (1 + float(rel) * 2.0 ** -24))))
            if 2 <= d < (1 << 24):
                out.append(d)
        if len(out) >= count:
            break
    return out


def band_ds(N: int, b: int) -> list:
    rng = np.random.default_rng(N + b)
    ds = [1, 2, 3, 64, 4095, 4096, 4097, (1 << 24) - 1, 1 << 24, 1 << 29]
    ds += [int(x) for x in rng.integers(2, 1 << 24, 12)]
    ds += near_threshold_ds(N, b, -7.0, 7.0, 10)
    return ds


def check_band(N: int, b: int, ds) -> bool:
    cm = np.array(ds, dtype=np.int64)
    mu_p = np.arange(len(ds), dtype=np.int64) % 7 - 3
    lo, hi = oz.mu_band(mu_p, cm, N, b)
    for i, d in enumerate(ds):
        el, eh = band_exact(int(d), N, b)
        if (lo[i], hi[i]) != (mu_p[i] + el, mu_p[i] + eh):
            return False
    return True


@pytest.mark.parametrize("b", [64, 32])
@pytest.mark.parametrize("N", [2, 9, 14, 17, 20, 33, 49])
def test_mu_band_exact(N, b):
    assert check_band(N, b, band_ds(N, b))


def test_mu_band_edges_are_reached():
    # the near-threshold cases include bands of width one (both floors occur),
    # so an evaluator that took only one end of the admissible e would fail
    widths = []
    for N in (9, 17, 33):
        for d in near_threshold_ds(N, 64, -3.0, 3.0, 10):
            el, eh = band_exact(d, N, 64)
            widths.append(eh - el)
    assert 1 in widths and 0 in widths


# --------------------------------------------------------------------------- #
# Planted mistakes (in the oracle, on the CPU): each must fail a pin above
# --------------------------------------------------------------------------- #
def _bt_variant(change):
    orig = oz.bound_terms

    def bt(N, b=64):
        d = dict(orig(N, b))
        change(d, N, b)
        return d
    return bt


def _t_of(P: int) -> float:
    return 1.0 / math.sqrt(32.0 * float(P)) * (1 + 2.0 ** -50)


PLANTS_T2 = {
    # t from P instead of P - 1
    "t_with_P": lambda d, N, b: d.update(t=_t_of(constants(N, b).P)),
    # t without its square root
    "t_no_sqrt": lambda d, N, b: d.update(t=1.0 / (32.0 * float(constants(N, b).P - 1))),
    # the k term counted twice
    "doubled_k": None,
    # R_b's P-proportional part without the factor 2^(1 + ceil(log2 rho))
    "gN_no_pow2": lambda d, N, b: d.update(gN=d["gN"] / 2.0 ** (1 + (constants(N, b).rho - 1).bit_length())
                                           if b == 64 else d["gN"]),
    # u |A'B'| instead of 3u |A'B'| (b = 64), and 1/2 u P instead of 3/2 u P in r_b
    "h_one_u": lambda d, N, b: d.update(h=d["h"] / 3.0 if b == 64 else d["h"],
                                        rb=d["rb"] - float(U64 * constants(N, b).P) if b == 64 else d["rb"]),
}


def _theorem2_all_cases() -> bool:
    for b in (64, 32):
        for N in NS:
            for case in CASES:
                A, B = case_inputs(case, N, b)
                if not check_theorem2(A, B, N, b):
                    return False
    return True


@pytest.mark.parametrize("plant", list(PLANTS_T2))
def test_planted_theorem2_mistakes_are_caught(monkeypatch, plant):
    if plant == "doubled_k":
        # (2k + ...) t^2 2^alpha' 2^beta': the k is added once more through both
        # constants that sit beside it
        orig = oz.bound_terms
        k_of = {}

        def bt(N, b=64):
            d = dict(orig(N, b))
            d["gN"] += k_of["k"]
            d["rb"] += k_of["k"]
            return d
        orig_bounds = oz.bounds

        def bounds(A, B, res):
            k_of["k"] = A.shape[1]
            return orig_bounds(A, B, res)
        monkeypatch.setattr(oz, "bound_terms", bt)
        monkeypatch.setattr(oz, "bounds", bounds)
    else:
        monkeypatch.setattr(oz, "bound_terms", _bt_variant(PLANTS_T2[plant]))
    assert not _theorem2_all_cases()


def test_planted_alpha_prime_mistakes_are_caught(monkeypatch):
    # 2^alpha' without sqrt(max cbar), and with max cbar where the paper has its square root
    orig = oz.pow2_prime
    monkeypatch.setattr(oz, "pow2_prime", lambda a, c: orig(a, np.minimum(c, 1)))
    assert not _theorem2_all_cases()
    monkeypatch.setattr(oz, "pow2_prime", lambda a, c: orig(a, np.asarray(c, np.int64) ** 2))
    assert not _theorem2_all_cases()


def test_planted_norm_mistake_is_caught(monkeypatch):
    # |A| v taken as the row maximum instead of the row sum
    monkeypatch.setattr(oz, "abs_sums", lambda X, axis: np.abs(np.asarray(X, np.float64)).max(axis=axis))
    assert not _theorem2_all_cases()
    assert not all(check_exponent_bound(*case_inputs(c, 8, 64), 8, 64) for c in CASES)


def test_planted_exponent_bound_mistakes_are_caught(monkeypatch):
    def all_ok():
        return all(check_exponent_bound(*case_inputs(c, N, b), N, b)
                   for b in (64, 32) for N in NS for c in CASES)
    monkeypatch.setattr(oz, "bound_terms", _bt_variant(PLANTS_T2["h_one_u"]))
    assert not all_ok()
    monkeypatch.setattr(oz, "bound_terms", _bt_variant(lambda d, N, b: d.update(gN=2 * d["gN"])))
    assert not all_ok()


def test_planted_splitk_mistakes_are_caught(monkeypatch, splitk_case):
    A, B, res = splitk_case
    orig = oz.bound_from_exponents
    # one range's bound counted at half its size
    monkeypatch.setattr(oz, "bound_from_exponents", lambda *a, **kw: 0.5 * orig(*a, **kw))
    assert not check_splitk(A, B, res, 64)
    monkeypatch.setattr(oz, "bound_from_exponents", orig)
    # the rounding of each addition left out: the partial sums taken as zero
    res0 = dict(res, partial=[np.zeros_like(p) for p in res["partial"]])
    got = oz.bound_splitk(A, B, res0, 64)
    x = splitk_bound_exact(A, B, res, 64)
    assert not all(within(got[i, j], (x[i][j], x[i][j])) for i in range(got.shape[0]) for j in range(got.shape[1]))


def test_planted_band_mistakes_are_caught(monkeypatch):
    def all_ok():
        return all(check_band(N, b, band_ds(N, b)) for b in (64, 32) for N in (2, 9, 14, 17, 20, 33, 49))
    # a band twice as wide (8 u32 log2 d)
    monkeypatch.setattr(oz, "U32", 2 * U32)
    assert not all_ok()
    monkeypatch.setattr(oz, "U32", U32)
    # round instead of floor
    monkeypatch.setattr(oz, "exponent_shift", lambda c, e, Pp: np.rint(
        np.float64(c) * e.astype(np.float64) + np.float64(Pp)).astype(np.int64))
    assert not all_ok()
