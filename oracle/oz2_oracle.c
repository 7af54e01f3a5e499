/*
 * Plain CPU oracle for the Ozaki-II scheme (arXiv 2602.02549).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library links, includes or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it (through ctypes, via oracle/ozaki2.py).
 *
 * Every routine here is a literal loop over the definition it names; there is
 * no blocking, vectorisation or reordering beyond what the definition states.
 * All floating-point work is IEEE binary64 (or binary32 where the paper says
 * single(.)), compiled with -ffp-contract=off so that every fused multiply-add
 * is an explicit fma() call.
 *
 * Matrices are addressed through (row stride, column stride) pairs so that the
 * same loop serves rows of A and columns of B.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Algorithm 2, lines for mu' and nu' (eq. mu'nu'):                          */
/*   mu'_i = 5 - floor(log2 max_h |a_ih|).                                   */
/* This routine returns floor(log2 max_h |x_ih|) (alpha_i of Theorem 2) for  */
/* each of `rows` vectors, or INT32_MIN for an all-zero vector.  frexp is    */
/* exact for every finite double, subnormals included:                      */
/*   x = f * 2^e with 0.5 <= |f| < 1  =>  floor(log2 |x|) = e - 1.           */
/* ------------------------------------------------------------------------- */
void oz2o_floor_log2_absmax(int rows, int cols, const double *X, long rs, long cs,
                            int32_t *out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < rows; i++) {
        double mx = 0.0;
        for (int h = 0; h < cols; h++) {
            double v = fabs(X[(long)i * rs + (long)h * cs]);
            if (v > mx) mx = v;
        }
        if (mx == 0.0) { out[i] = INT32_MIN; continue; }
        int e;
        (void)frexp(mx, &e);
        out[i] = e - 1;
    }
}

/* Algorithm 2, lines for Abar and Bbar:  xbar_ih = ceil(2^shift_i |x_ih|).   */
/* ldexp is exact unless the result underflows; a nonzero x whose scaled      */
/* value underflows to zero still has ceil(.) = 1, which is set explicitly.   */
void oz2o_ceil_scaled_abs(int rows, int cols, const double *X, long rs, long cs,
                          const int32_t *shift, int8_t *out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < rows; i++) {
        for (int h = 0; h < cols; h++) {
            double a = fabs(X[(long)i * rs + (long)h * cs]);
            double v;
            if (a == 0.0) v = 0.0;
            else {
                v = ceil(ldexp(a, shift[i]));
                if (v < 1.0) v = 1.0;
            }
            out[(long)i * cols + h] = (int8_t)v;   /* 0 <= v <= 64 */
        }
    }
}

/* Z = X * Y with X (m x k) and Y (k x n) int8 row-major, Z int64 row-major:  */
/* the exact integer matrix product (Algorithm 2 Cbar = Abar Bbar; Algorithm  */
/* 3 C'_l = A'_l B'_l, here without the INT32 wrap, which does not change the */
/* residue modulo p_l).                                                       */
void oz2o_gemm_i8_i64(int m, int n, int k, const int8_t *X, const int8_t *Y, int64_t *Z)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; i++) {
        int64_t *z = Z + (long)i * n;
        for (int j = 0; j < n; j++) z[j] = 0;
        for (int h = 0; h < k; h++) {
            int64_t a = X[(long)i * k + h];
            if (a == 0) continue;
            const int8_t *y = Y + (long)h * n;
            for (int j = 0; j < n; j++) z[j] += a * (int64_t)y[j];
        }
    }
}

/* Algorithm 2, lines for A' and B':  x'_ih = trunc(2^shift_i * x_ih).        */
void oz2o_trunc_scaled(int rows, int cols, const double *X, long rs, long cs,
                       const int32_t *shift, double *out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < rows; i++)
        for (int h = 0; h < cols; h++)
            out[(long)i * cols + h] = trunc(ldexp(X[(long)i * rs + (long)h * cs], shift[i]));
}

/* mod(x, p) := x - p*round(x/p) (Section 1.2), stored as INT8.  fmod is     */
/* exact for doubles.  For p = 256 the class of 128 is stored as -128, which  */
/* is what a cast to INT8 produces (Section 3.1).                             */
static int8_t balanced_from_remainder(double r, int p)
{
    /* r = x - p*trunc(x/p), |r| < p */
    if (r > 0.5 * p) r -= p;
    else if (r < -0.5 * p) r += p;
    if (p == 256 && r == 128.0) r = -128.0;
    return (int8_t)r;
}

void oz2o_residues(long count, const double *X, int p, int8_t *out)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < count; i++)
        out[i] = balanced_from_remainder(fmod(X[i], (double)p), p);
}

/* Algorithm 3, W_l = mod(C'_l, p_l) stored as INT8.                          */
void oz2o_mod_i64(long count, const int64_t *X, int p, int8_t *out)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < count; i++) {
        int64_t r = X[i] % p;                   /* sign of X[i], |r| < p */
        if (2 * r > p) r -= p;
        else if (2 * r < -p) r += p;
        if (p == 256 && r == 128) r = -128;
        out[i] = (int8_t)r;
    }
}

/* Algorithm 1, last line: C = fl(diag(2^-mu) C'' diag(2^-nu)), taken as one   */
/* scaling by 2^-(mu_i + nu_j) (a single rounding, which only matters when    */
/* the result is subnormal).  b = 32: C = single(2^-(mu_i+nu_j) C''), the     */
/* FP64 scaling being exact wherever the FP32 result is not zero.             */
void oz2o_unscale(int m, int n, const double *Cpp, const int32_t *mu, const int32_t *nu,
                  int b, double *C)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) {
            long e = (long)i * n + j;
            int s = -(mu[i] + nu[j]);
            if (b == 32) C[e] = (double)(float)ldexp(Cpp[e], s);
            else C[e] = ldexp(Cpp[e], s);
        }
}

/* Algorithm 2, e_i = log2f(max_h dbar_ih): the C library's log2f.            */
void oz2o_log2f(long count, const float *x, float *out)
{
    for (long i = 0; i < count; i++) out[i] = log2f(x[i]);
}

/* ------------------------------------------------------------------------- */
/* Exact dot products (for the error of C against the exact product AB).     */
/*                                                                           */
/* A fixed-point two's-complement integer of NL 64-bit limbs whose bit 0     */
/* weighs 2^EMIN holds sum_h a_h b_h - c exactly: every double is M * 2^E    */
/* with |M| < 2^53 and E >= -1074, so a product is an integer below 2^106    */
/* times 2^(Ea+Eb) with Ea+Eb >= -2148 - 106 + 106.  The sum is rounded to   */
/* the nearest double (ties to even) once, at the end.                       */
/* ------------------------------------------------------------------------- */
#define EMIN (-2304)
#define NL 72                 /* 4608 bits: 2^-2304 .. 2^2303, sign included */

typedef struct { uint64_t l[NL]; } bigfix;

static void big_add_mag(bigfix *x, unsigned __int128 mag, int shift, int negative)
{
    /* add (or subtract) mag * 2^shift (shift >= 0) */
    int li = shift >> 6, bo = shift & 63;
    uint64_t w[4] = {0, 0, 0, 0};
    uint64_t lo = (uint64_t)mag, hi = (uint64_t)(mag >> 64);
    if (bo == 0) { w[0] = lo; w[1] = hi; }
    else {
        w[0] = lo << bo;
        w[1] = (lo >> (64 - bo)) | (hi << bo);
        w[2] = hi >> (64 - bo);
    }
    if (!negative) {
        unsigned carry = 0;
        for (int t = 0; li + t < NL; t++) {
            uint64_t add = t < 4 ? w[t] : 0;
            if (t >= 4 && carry == 0) break;
            unsigned __int128 s = (unsigned __int128)x->l[li + t] + add + carry;
            x->l[li + t] = (uint64_t)s;
            carry = (unsigned)(s >> 64);
        }
    } else {
        unsigned borrow = 0;
        for (int t = 0; li + t < NL; t++) {
            uint64_t sub = t < 4 ? w[t] : 0;
            if (t >= 4 && borrow == 0) break;
            uint64_t a = x->l[li + t];
            unsigned __int128 d = (unsigned __int128)a - sub - borrow;
            x->l[li + t] = (uint64_t)d;
            borrow = (unsigned)((d >> 64) != 0);
        }
    }
}

static void decompose(double v, int64_t *M, int *E)
{
    /* v = M * 2^E exactly, |M| < 2^53 */
    int e;
    double f = frexp(v, &e);
    *M = (int64_t)ldexp(f, 53);
    *E = e - 53;
}

static void big_add_product(bigfix *x, double a, double b)
{
    if (a == 0.0 || b == 0.0) return;
    int64_t Ma, Mb; int Ea, Eb;
    decompose(a, &Ma, &Ea);
    decompose(b, &Mb, &Eb);
    int neg = (Ma < 0) != (Mb < 0);
    unsigned __int128 mag = (unsigned __int128)(uint64_t)llabs(Ma) * (uint64_t)llabs(Mb);
    big_add_mag(x, mag, Ea + Eb - EMIN, neg);
}

static void big_add_double(bigfix *x, double c, int negate)
{
    if (c == 0.0) return;
    int64_t M; int E;
    decompose(c, &M, &E);
    int neg = (M < 0) != (negate != 0);
    big_add_mag(x, (unsigned __int128)(uint64_t)llabs(M), E - EMIN, neg);
}

static int big_bit(const bigfix *x, int pos)
{
    return (int)((x->l[pos >> 6] >> (pos & 63)) & 1u);
}

static double big_to_double(bigfix *x)
{
    int neg = (int)(x->l[NL - 1] >> 63);
    if (neg) {                     /* two's-complement negate */
        unsigned carry = 1;
        for (int t = 0; t < NL; t++) {
            unsigned __int128 s = (unsigned __int128)(~x->l[t]) + carry;
            x->l[t] = (uint64_t)s;
            carry = (unsigned)(s >> 64);
        }
    }
    int top = -1;
    for (int t = NL - 1; t >= 0; t--)
        if (x->l[t]) { top = t * 64 + 63 - __builtin_clzll(x->l[t]); break; }
    if (top < 0) return 0.0;
    /* exponent of the leading bit, and of the result's last kept bit */
    int elead = top + EMIN;
    int elsb = elead - 52;
    if (elsb < -1074) elsb = -1074;             /* subnormal result */
    int d = elsb - EMIN;                        /* bit index of the kept LSB */
    uint64_t kept = 0;
    for (int pos = top; pos >= d; pos--) kept = (kept << 1) | (uint64_t)big_bit(x, pos);
    int roundbit = d - 1 >= 0 ? big_bit(x, d - 1) : 0;
    int sticky = 0;                             /* any bit below the round bit */
    if (d - 2 >= 0) {
        int top_limb = (d - 2) >> 6, nb = ((d - 2) & 63) + 1;
        uint64_t mask = nb == 64 ? ~0ull : ((1ull << nb) - 1);
        sticky = (x->l[top_limb] & mask) != 0;
        for (int t = 0; t < top_limb && !sticky; t++) sticky = x->l[t] != 0;
    }
    if (roundbit && (sticky || (kept & 1u))) kept++;
    double r = ldexp((double)kept, elsb);
    return neg ? -r : r;
}

/* Algorithm 3, accumulation and final reduction, per entry:                  */
/*   C'(1) = fl(sum_l s_l1 W_l),  C'(2) = fl(sum_l s_l2 W_l),                   */
/*   Q = round(fl(P_inv * C'(1))),                                             */
/*   C'' = fl(fma(-Q, P2, fma(-Q, P1, C'(1)) + C'(2))).                        */
/* Reading of fl(sum): each sum is taken exactly and rounded to the nearest   */
/* double once.  The Section 4 analysis (proof of Lemma 2) bounds the error   */
/* of any floating-point evaluation of these sums by N u_64 sum |s_l2 W_l|;   */
/* the correctly rounded sum meets that bound and is the one evaluation whose */
/* value does not depend on the order of the terms.  For b = 64, C'(1) is     */
/* exact (Lemma 2), so only C'(2) is affected; for b = 32, s_l2 = 0 and       */
/* C'(1) is the rounded sum.                                                  */
/* fma_chain != 0 selects the other reading instead: both sums as fma chains  */
/* in ascending l from +0 (an FP64 evaluation in one fixed order).            */
/* For b = 32 the rounding C'' = single(C'') is taken after the inverse        */
/* scaling (oz2o_unscale), where it gives the same value whenever single(C'')  */
/* is finite and C is normal, and does not overflow when P > 2^128.            */
/* W holds N planes of `count` entries.                                        */
void oz2o_crt(long count, int N, const int8_t *W, const double *s1, const double *s2,
              double P1, double P2, double Pinv, int b, int fma_chain,
              double *C1out, double *C2out, double *Qout, double *Cpp)
{
#pragma omp parallel for schedule(static)
    for (long e = 0; e < count; e++) {
        double c1 = 0.0, c2 = 0.0;
        if (fma_chain) {
            for (int l = 0; l < N; l++) {
                double w = (double)W[(long)l * count + e];
                c1 = fma(s1[l], w, c1);
                c2 = fma(s2[l], w, c2);
            }
        } else {
            bigfix a1, a2;
            memset(&a1, 0, sizeof a1);
            memset(&a2, 0, sizeof a2);
            for (int l = 0; l < N; l++) {
                double w = (double)W[(long)l * count + e];
                big_add_product(&a1, s1[l], w);
                big_add_product(&a2, s2[l], w);
            }
            c1 = big_to_double(&a1);
            c2 = big_to_double(&a2);
        }
        double q = nearbyint(Pinv * c1);        /* round to nearest (even) */
        double c = fma(-q, P2, fma(-q, P1, c1) + c2);
        (void)b;
        if (C1out) C1out[e] = c1;
        if (C2out) C2out[e] = c2;
        if (Qout) Qout[e] = q;
        Cpp[e] = c;
    }
}

/* out_ij = RN( sum_h X[i,h] Y[h,j] - (Cm ? Cm[i,j] : 0) ), computed exactly   */
/* and rounded once.  X is addressed (i, h) -> X[i*xr + h*xc], Y (h, j) ->     */
/* Y[h*yr + j*yc], Cm and out are m x n row-major.                            */
void oz2o_exact_residual(int m, int n, int k, const double *X, long xr, long xc,
                         const double *Y, long yr, long yc, const double *Cm, double *out)
{
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) {
            bigfix acc;
            memset(&acc, 0, sizeof acc);
            for (int h = 0; h < k; h++)
                big_add_product(&acc, X[(long)i * xr + (long)h * xc], Y[(long)h * yr + (long)j * yc]);
            if (Cm) big_add_double(&acc, Cm[(long)i * n + j], 1);
            out[(long)i * n + j] = big_to_double(&acc);
        }
}

/* Exact rounded sums sum_h |x_ih| (for the |A| v and v^T |B| terms).         */
void oz2o_exact_abs_sums(int rows, int cols, const double *X, long rs, long cs, double *out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < rows; i++) {
        bigfix acc;
        memset(&acc, 0, sizeof acc);
        for (int h = 0; h < cols; h++) big_add_double(&acc, fabs(X[(long)i * rs + (long)h * cs]), 0);
        out[i] = big_to_double(&acc);
    }
}

int oz2o_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
