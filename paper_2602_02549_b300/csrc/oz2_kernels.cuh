// Device code of the Ozaki-II path (arXiv 2602.02549) for sm_103a.
//
// Included once, by oz2_api.cu, so that the __constant__ tables below live in a
// single translation unit with every kernel that reads them.
//
//   k_absmax                  Algorithm 2 inputs: max |x| per row of A (per
//                             column of B) -> mu', nu', and the per-k maxima
//                             of the N rule (one HBM read)
//   k_quant_kc / k_quant_rc   Abar = ceil(2^mu' |A|), Bbar likewise, as BF16
//   (k_quant: both)           (K-contiguous rows, or transposed through shared
//                             memory); also |A| v and v^T |B| for the N rule
//   k_gemm<EPI_MAX>           Cbar = Abar Bbar on tcgen05, keeping only the row
//                             and column maxima of Cbar
//   k_bound, k_exponents      the N rule; Dbar, e, f, mu, nu (Algorithm 2)
//   k_resid_kc / k_resid_rc   A'_l = mod(trunc(2^mu A), p_l) as BF16, N planes
//   k_gemm<EPI_MOD>           C'_l = A'_l B'_l on tcgen05, W_l = mod(C'_l, p_l)
//   k_crt                     C'(1), C'(2), Q, C'' (Algorithm 3) and the
//                             inverse scaling of Algorithm 1
#pragma once
#include <cuda_bf16.h>
#include <climits>
#include <cstdint>
#include <type_traits>

#include "oz2_ptx.cuh"
#include "oz2_tables.h"

namespace oz2 {

// ============================================================= constant tables
struct DevN {
    double P1, P2, Pinv, g, t, gN;
    float Pprime;
    int eg;       // b = 64: g = 2^eg
    int esum;     // grid exponent of the rounded CRT sum
    int poff;     // first plane pair of this N in c_dp64 / c_dp32
    long long M1; // b = 64: P1 = M1 2^eu1, g = 2^(eu1 + sh)
    int eu1, sh;
    int kq, sq;   // b = 64: (H >> 22) kq 2^-sq estimates H g / P
};

__constant__ DevN c_n64[kNMax + 1];
__constant__ DevN c_n32[kNMax + 1];
// CRT constants as 16-bit pieces, two planes per word (Tables::dp64 / dp32)
__constant__ uint4 c_dp64[kPairsLen][2];  // b = 64: pieces 0-3 of s_l1 / g, then of s_l2 / 2^esum
__constant__ uint4 c_dp32[kPairsLen];     // b = 32: pieces 0-3 of s_l1 / 2^esum
__constant__ float c_cneg;                 // single_down(-0.5/(1-4 u32))
__constant__ float c_w12[kNMax][kLimbs];   // balanced 2^(12 j) mod p_l
// per modulus, each value duplicated into both FP32 lanes: balanced
// 2^(13 j) mod p_l (j < 8), RN(1/p_l), -p_l
__constant__ unsigned long long c_w13p[kNMax][kFixLimbs + 2];
__device__ uint8_t g_pow2[kNMax][256];     // 2^E mod p_l
__constant__ float c_pf[kNMax];            // p_l
__constant__ float c_invp[kNMax];          // RN_f32(1/p_l)

// Device status word: bit 0 = a bounded wait expired.
__device__ int g_status;

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per wait

// ============================================================= small helpers
// floor(log2 x) of a positive double given by its bits.
__device__ __forceinline__ int floor_log2_bits(uint64_t b) {
    int ex = int(b >> 52);
    if (ex) return ex - 1023;
    uint64_t m = b & ((1ull << 52) - 1);
    return -1074 + (63 - __clzll((long long)m));
}

// x = (-1)^neg * M * 2^e with M an integer (< 2^53), from the bits of x.
struct Split {
    uint64_t M;
    int e;
    bool neg;
};
__device__ __forceinline__ Split split_bits(double x) {
    uint64_t b = (uint64_t)__double_as_longlong(x);
    Split s;
    s.neg = (b >> 63) != 0;
    int ex = int((b >> 52) & 0x7FF);
    uint64_t man = b & ((1ull << 52) - 1);
    if (ex == 0) { s.M = man; s.e = -1074; }
    else { s.M = man | (1ull << 52); s.e = ex - 1075; }
    if (ex == 0x7FF) s.M = 0;                  // non-finite: precondition violated
    return s;
}
__device__ __forceinline__ Split split_bits(float x) {
    uint32_t b = __float_as_uint(x);
    Split s;
    s.neg = (b >> 31) != 0;
    int ex = int((b >> 23) & 0xFF);
    uint32_t man = b & ((1u << 23) - 1);
    if (ex == 0) { s.M = man; s.e = -149; }
    else { s.M = man | (1u << 23); s.e = ex - 150; }
    if (ex == 0xFF) s.M = 0;
    return s;
}

// Algorithm 2: xbar = ceil(2^shift |x|), 0 <= xbar <= 64 for shift = 5 - floor(log2 max).
template <typename T>
__device__ __forceinline__ uint32_t ceil_scaled_abs(T x, int shift) {
    Split s = split_bits(x);
    if (s.M == 0) return 0;
    int sh = s.e + shift;
    if (sh >= 0) return sh > 10 ? 127u : uint32_t(s.M << sh);
    int r = -sh;
    if (r >= 64) return 1;
    uint64_t q = s.M >> r;
    return uint32_t(q + ((s.M & ((1ull << r) - 1)) != 0));
}

// floor(2^shift |x|) (the componentwise N rule's lower bound of 2^shift |x|).
template <typename T>
__device__ __forceinline__ uint32_t floor_scaled_abs(T x, int shift) {
    Split s = split_bits(x);
    if (s.M == 0) return 0;
    int sh = s.e + shift;
    if (sh >= 0) return sh > 10 ? 127u : uint32_t(s.M << sh);
    const int r = -sh;
    return r >= 64 ? 0u : uint32_t(s.M >> r);
}

// Algorithm 2: x' = trunc(2^shift x) = (-1)^neg * M * 2^E, E >= 0.
struct Int {
    uint64_t M;
    int E;
    bool neg;
};
template <typename T>
__device__ __forceinline__ Int trunc_scaled(T x, int shift) {
    Split s = split_bits(x);
    Int v;
    v.neg = s.neg;
    int sh = s.e + shift;
    if (sh >= 0) { v.M = s.M; v.E = sh; }
    else { v.M = (-sh >= 64) ? 0 : (s.M >> (-sh)); v.E = 0; }
    return v;
}

// Residues of x' = trunc(2^shift x) (Algorithm 3, A'_l = mod(A', p_l)).
// x' = (-1)^neg M 2^E with M < 2^53.  M is cut once into five 12-bit limbs d_i
// (with the sign of x'); for odd p_l and balanced weights w_i = 2^(12 i) mod p_l
// in [-(p-1)/2, (p-1)/2]:
//   t  = sum_i d_i w_i,  |t| < 5 * 2^12 * 127 < 2^22, exact in FP32 (every
//        product and partial sum is an integer below 2^24);
//   r1 = t - p rint(t / p),    balanced residue of M (with sign);
//   v  = r1 (2^E mod p_l),     |v| < 2^15, exact;
//   r  = v - p rint(v / p),    the balanced residue of x'.
// rint(t * RN(1/p)) equals round(t / p) because t / p lies at least 1/(2p) from
// a half-integer (p odd) while the FP32 error is below |t| 2^-23 / p < 1/(2p).
// p = 256 takes the low byte of x' in two's complement (class 128 -> -128).
struct Limbs {
    float d[kLimbs];
    int E;       // table index (clamped to 255)
    int r256;    // residue modulo 256
};

template <typename T>
__device__ __forceinline__ Limbs limbs_of(T x, int shift) {
    const Int v = trunc_scaled(x, shift);
    const uint32_t lo = uint32_t(v.M), hi = uint32_t(v.M >> 32);
    const uint32_t e[kLimbs] = {lo & 0xFFFu, (lo >> 12) & 0xFFFu, ((lo >> 24) | (hi << 8)) & 0xFFFu,
                                (hi >> 4) & 0xFFFu, (hi >> 16) & 0xFFFu};
    Limbs L;
#pragma unroll
    for (int i = 0; i < kLimbs; i++) L.d[i] = v.neg ? -float(e[i]) : float(e[i]);
    L.E = v.E > 255 ? 255 : v.E;
    uint32_t b = v.E >= 8 ? 0u : ((lo << v.E) & 255u);
    if (v.neg) b = (256u - b) & 255u;
    L.r256 = int(int8_t(b));
    return L;
}

__device__ __forceinline__ float residue_odd(const Limbs &L, int l, const uint8_t (*pow2)[256]) {
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < kLimbs; i++) t = fmaf(L.d[i], c_w12[l][i], t);
    const float p = c_pf[l], ip = c_invp[l];
    const float r1 = fmaf(-rintf(t * ip), p, t);
    const float v = r1 * float(pow2[l][L.E]);
    return fmaf(-rintf(v * ip), p, v);
}

__device__ __forceinline__ uint32_t pack_bf16x2f(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// ============================================================= operand views
// Logical matrix X[r][h], r < R, h < k: A rows (r = i) or B columns (r = j).
// kcontig: element at ptr[r*ld + h]; else at ptr[h*ld + r].
template <typename T>
struct Operand {
    const T *ptr;
    long ld;
    int R;
    int kcontig;
};

// ============================================================= grouped launches
// Every phase outside the two GEMMs runs as one launch over the work items of
// all problems of a group: one problem for oz2_gemm_ex, up to kMaxJobs for a
// batch.  Blocks walk the items g = blockIdx.x, blockIdx.x + gridDim.x, ...;
// problem p owns the items [begin[p], begin[p+1]).  The item counts below are
// shared by the host (which fills begin[]) and the kernels (which decode).
constexpr int kMaxJobs = 64;
constexpr int kLineBlock = 64;     // lines per k_absmax item, unless the launch has few items

template <typename T>
struct JobDesc {
    Operand<T> op[2];              // A (logical rows i) and B (logical rows j)
    T *C;
    long ldc;
    int m, n, k, k_pad, n_pad;
    int R_pad[2];                  // m_pad, n_pad
    int nmoduli, nmax, fast, inject, vec[2];
    int cw;                        // componentwise N rule (OZ2_COMPONENTWISE)
    int absmax_lb;                 // lines per k_absmax item (kLineBlock or fewer, per launch)
    int absmax_lw[2];              // line groups per k_absmax block (1, 2, 4 or 8), per operand
    int accum;                     // CRT adds its result to C (the K ranges after the first)
    double target;
    unsigned long long *hmax[2];   // per-k maxima of |A|, |B|
    unsigned long long *rmax[2];   // per logical row maxima (bits)
    unsigned long long *l1[2];     // fixed-point 1-norms (PlaneArgs::l1)
    unsigned long long *red;       // bound reductions
    float *cwv[2];                 // componentwise rule: (R_i 2^mu'_i, 2^alpha'_i 2^mu'_i) per row of A,
                                   // (2^beta'_j 2^nu'_j, K_j 2^nu'_j) per column of B, rounded up
    int *cmax[2];                  // Cbar row / column maxima
    int *ss[2];                    // fast mode: sums of squares of Abar rows / Bbar columns
    int *ndev, *n_out;
    int32_t *expo[2];              // mu, nu computed by k_exponents
    const int32_t *shift[2];       // mu, nu as used (computed or injected)
    int32_t *expo_out[2];          // optional exports
    __nv_bfloat16 *res[2];
    long plane[2];
    int8_t *W;
    long w_plane;
    uint4 *zero;                   // region cleared at the start of a call
    long zero_vec;                 // its size in 16-byte units
};

// CAP: problems the table holds (1 for a single call, so that each launch
// passes a small parameter; kMaxJobs for a batch)
template <typename T, int CAP = kMaxJobs>
struct JobGroup {
    JobDesc<T> j[CAP];
    int count;
    long long begin[CAP + 1];
};

__host__ __device__ __forceinline__ long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

// k_absmax: operand X stored as S lines of C contiguous elements
template <typename T>
__host__ __device__ __forceinline__ void absmax_geom(const JobDesc<T> &j, int X, int &S, int &C) {
    if (j.op[X].kcontig) { S = j.op[X].R; C = j.k; }
    else { S = j.k; C = j.op[X].R; }
}
// k_absmax item: j.absmax_lb lines x 256 (8 / lw) positions, lw = j.absmax_lw[X]
// line groups: a warp covers 256 positions of a line (8 per lane), the block's
// 8 warps form 8 / lw position groups times lw line groups, and each line
// group takes every lw-th line of the item.
template <typename T>
__host__ __device__ __forceinline__ long long items_absmax_x(const JobDesc<T> &j, int X) {
    if (j.inject) return 0;
    int S, C;
    absmax_geom(j, X, S, C);
    return cdiv(S, j.absmax_lb) * cdiv(C, 2048 / j.absmax_lw[X]);
}
// the item width for lines of C positions: the one that leaves the fewest idle
// positions (the host may narrow it further for small launches)
__host__ __device__ __forceinline__ int absmax_lw_min(int C) {
    // the fewest positions past C over the item columns (ties: fewer line
    // groups, i.e. wider items)
    int best = 8;
    long long least = -1;
    for (int lw = 8; lw >= 1; lw >>= 1) {
        const long long pw = 2048 / lw;
        const long long waste = cdiv(C, pw) * pw - C;
        if (least < 0 || waste <= least) { least = waste; best = lw; }
    }
    return best;
}
// Residues of K-contiguous rows: 256 consecutive groups of 8 positions per
// item, in the row-major order of the plane's R live rows of k_pad positions
// (R x k_pad / 8 groups in all; the last item may end early).  Transposed
// rows: 16 x 128 tiles over the R live rows.
template <typename T>
__host__ __device__ __forceinline__ long long items_kc_x(const JobDesc<T> &j, int X) {
    if (!j.op[X].kcontig) return 0;
    return cdiv((long long)j.op[X].R * (j.k_pad / 8), 256);
}
template <typename T>
__host__ __device__ __forceinline__ long long items_rc_x(const JobDesc<T> &j, int X) {
    return j.op[X].kcontig ? 0 : cdiv(j.k_pad, 128) * cdiv(j.op[X].R, 16);
}
// quantisation of K-contiguous rows: kQuantGroups chunks of tpr x 8 h per item;
// tpr is a power of two in [8, 256] with tpr x 8 x kQuantGroups >= k_pad where
// possible, so that short rows share a block (and a warp) instead of leaving
// threads idle
constexpr int kQuantGroups = 4;
__host__ __device__ __forceinline__ int quant_tpr(int k_pad) {
    // the width whose items leave the fewest h positions past k_pad (ties: the
    // wider, with fewer items per row and so fewer atomic row sums)
    int best = 8;
    long long least = -1;
    for (int t = 8; t <= 256; t <<= 1) {
        const long long per = (long long)t * 8 * kQuantGroups;
        const long long waste = cdiv(k_pad, per) * per - k_pad;
        if (least < 0 || waste <= least) { least = waste; best = t; }
    }
    return best;
}
template <typename T>
__host__ __device__ __forceinline__ long long items_quant_kc_x(const JobDesc<T> &j, int X) {
    if (j.inject || !j.op[X].kcontig) return 0;
    const int tpr = quant_tpr(j.k_pad);
    return cdiv(j.R_pad[X], 256 / tpr) * cdiv(j.k_pad, tpr * 8 * kQuantGroups);
}
template <typename T>
__host__ __device__ __forceinline__ long long items_quant_rc_x(const JobDesc<T> &j, int X) {
    // every row of R_pad: the scaling GEMM's maxima need zeros in the padding
    return j.inject || j.op[X].kcontig ? 0 : (long long)(j.k_pad / 64) * (j.R_pad[X] / 64);
}

template <typename T> struct Items {
    __host__ __device__ static long long clear(const JobDesc<T> &j) { return cdiv(j.zero_vec, 256); }
    __host__ __device__ static long long absmax(const JobDesc<T> &j) {
        return items_absmax_x(j, 0) + items_absmax_x(j, 1);
    }
    __host__ __device__ static long long quant_kc(const JobDesc<T> &j) {
        return items_quant_kc_x(j, 0) + items_quant_kc_x(j, 1);
    }
    __host__ __device__ static long long quant_rc(const JobDesc<T> &j) {
        return items_quant_rc_x(j, 0) + items_quant_rc_x(j, 1);
    }
    __host__ __device__ static long long fast_max(const JobDesc<T> &j) {
        return j.fast && !j.inject ? cdiv(j.m > j.n ? j.m : j.n, 2048) : 0;
    }
    __host__ __device__ static long long fast_cmax(const JobDesc<T> &j) {
        return j.fast && !j.inject ? cdiv(j.m + j.n, 2048) : 0;
    }
    __host__ __device__ static long long bound(const JobDesc<T> &j) {
        const int mx = j.m > j.n ? (j.m > j.k ? j.m : j.k) : (j.n > j.k ? j.n : j.k);
        return !j.inject && j.nmoduli == 0 ? cdiv(mx, 256) : 0;
    }
    __host__ __device__ static long long exponents(const JobDesc<T> &j) { return cdiv(j.m + j.n, 256); }
    __host__ __device__ static long long resid_kc(const JobDesc<T> &j) { return items_kc_x(j, 0) + items_kc_x(j, 1); }
    __host__ __device__ static long long resid_rc(const JobDesc<T> &j) { return items_rc_x(j, 0) + items_rc_x(j, 1); }
    __host__ __device__ static long long quant(const JobDesc<T> &j) { return quant_kc(j) + quant_rc(j); }
    __host__ __device__ static long long crt(const JobDesc<T> &j) {
        return cdiv((long long)j.m * cdiv(j.n, 4), 256);
    }
};

// Calls f(job, local item) for this block's items, in increasing order.
template <typename T, int CAP, class F>
__device__ __forceinline__ void for_items(const JobGroup<T, CAP> &G, F &&f) {
    const long long total = G.begin[G.count];
    int p = 0;
    if (CAP > 1 && blockIdx.x < total) {     // the first item's problem by bisection
        int hi = G.count - 1;
        while (p < hi) {
            const int mid = (p + hi + 1) >> 1;
            if (G.begin[mid] <= (long long)blockIdx.x) p = mid;
            else hi = mid - 1;
        }
    }
    for (long long g = blockIdx.x; g < total; g += gridDim.x) {
        while (G.begin[p + 1] <= g) p++;
        f(G.j[p], g - G.begin[p]);
    }
}

template <typename T, int CAP>
__global__ void __launch_bounds__(256) k_clear(const __grid_constant__ JobGroup<T, CAP> G) {
    for_items(G, [&](const JobDesc<T> &j, long long li) {
        const long long v = li * 256 + threadIdx.x;
        if (v < j.zero_vec) j.zero[v] = make_uint4(0, 0, 0, 0);
    });
}

// ============================================================= stats
// Maxima of |x| (as the bits of double(|x|), which order like the values)
// over an operand stored as S lines of C contiguous elements: per line and per
// position, merged with atomicMax (so the result does not depend on the
// order).  A, K-contiguous: lines are rows i, positions h.  B, R-contiguous:
// lines are h, positions are columns j.
template <typename T>
__device__ __forceinline__ unsigned long long abs_bits(T x) {
    return (unsigned long long)__double_as_longlong(fabs(double(x)));
}
template <>
__device__ __forceinline__ unsigned long long abs_bits<double>(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    const unsigned hi = __reduce_max_sync(0xffffffffu, unsigned(v >> 32));
    const unsigned lo = __reduce_max_sync(0xffffffffu, unsigned(v >> 32) == hi ? unsigned(v) : 0u);
    return ((unsigned long long)hi << 32) | lo;
}

// Item: j.absmax_lb lines x PW = 256 (8 / lw) positions of one operand (see
// items_absmax_x).  Each line's maximum over the item is one atomicMax per
// warp; each position's maximum over the item's lines is reduced across the
// lw line groups through shared memory first, so that a position takes one
// atomicMax per item.
template <typename T, int CAP>
__global__ void __launch_bounds__(256) k_absmax(const __grid_constant__ JobGroup<T, CAP> G) {
    __shared__ unsigned long long part[2048];   // [line group][position group][e 32 + lane]
    for_items(G, [&](const JobDesc<T> &j, long long li) {
        int X = 0;
        const long long n0 = items_absmax_x(j, 0);
        if (li >= n0) { X = 1; li -= n0; }
        int S, C;
        absmax_geom(j, X, S, C);
        const int lw = j.absmax_lw[X], npg = 8 / lw, PW = 256 * npg;
        const unsigned ncb = unsigned(cdiv(C, PW)), ui = unsigned(li);
        const int lb = int(ui / ncb), cb = int(ui - unsigned(lb) * ncb);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int pg = warp % npg, lg = warp / npg;
        const int c0 = cb * PW + pg * 256 + lane * 8;
        const int LB = j.absmax_lb;
        const int s_end = min(S, (lb + 1) * LB);
        const bool kc = j.op[X].kcontig != 0;
        unsigned long long *smax = kc ? j.rmax[X] : j.hmax[X];
        unsigned long long *cmax = kc ? j.hmax[X] : j.rmax[X];
        const T *ptr = j.op[X].ptr;
        const long ld = j.op[X].ld;
        const bool full = c0 + 8 <= C, vec = full && j.vec[X];
        unsigned long long cm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int s = lb * LB + lg; s < s_end; s += lw) {
            const T *src = ptr + (long)s * ld + c0;
            T x[8];
            if (vec) {
                if constexpr (sizeof(T) == 8) {
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const double2 v = reinterpret_cast<const double2 *>(src)[q];
                        x[2 * q] = T(v.x);
                        x[2 * q + 1] = T(v.y);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        const float4 v = reinterpret_cast<const float4 *>(src)[q];
                        x[4 * q] = T(v.x); x[4 * q + 1] = T(v.y); x[4 * q + 2] = T(v.z); x[4 * q + 3] = T(v.w);
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; e++) x[e] = c0 + e < C ? src[e] : T(0);
            }
            unsigned long long lm = 0;
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const unsigned long long bits = abs_bits(x[e]);
                cm[e] = bits > cm[e] ? bits : cm[e];
                lm = bits > lm ? bits : lm;
            }
            lm = warp_max_u64(lm);
            if (lane == 0 && lm) atomicMax(smax + s, lm);
        }
        if (lw == 1) {                       // one line group: no reduction across warps
#pragma unroll
            for (int e = 0; e < 8; e++)
                if (cm[e] && c0 + e < C) atomicMax(cmax + c0 + e, cm[e]);
            return;
        }
        __syncthreads();                     // the previous item's reads of part are done
#pragma unroll
        for (int e = 0; e < 8; e++) part[lg * PW + pg * 256 + e * 32 + lane] = cm[e];
        __syncthreads();
        // thread t: positions u 256 + t of the item (u < npg), position q = t of
        // position group u stored at u 256 + (q % 8) 32 + q / 8
        const int t = threadIdx.x, slot = (t & 7) * 32 + (t >> 3);
        for (int u = 0; u < npg; u++) {
            unsigned long long v = 0;
            for (int g = 0; g < lw; g++) {
                const unsigned long long w = part[g * PW + u * 256 + slot];
                v = w > v ? w : v;
            }
            const int c = cb * PW + u * 256 + t;
            if (v && c < C) atomicMax(cmax + c, v);
        }
    });
}

// ============================================================= planes
// k_quant_*: Abar = BF16(ceil(2^mu' |x|)), plane 0, K-major, zeros in the padding.
// k_resid_*: planes l < N = BF16(mod(trunc(2^mu x), p_l)), K-major, zeros past k in
// each row; rows R .. R_pad-1 are not written (a padded row of A'_l or B'_l
// reaches only rows or columns of C'_l past m or n, which the CRT never reads).
// Output element (l, r, h) at out[l*plane + r*k_pad + h].
struct PlaneArgs {
    __nv_bfloat16 *out;
    long plane;          // elements between planes
    int R_pad, k, k_pad;
    const unsigned long long *row_max;   // quantisation: shift = 5 - floor(log2 max)
    const int32_t *shift;                 // residues: mu or nu
    const int *n_dev;                     // residues: number of planes
    int *sumsq;                           // quantisation, fast mode: sum_h xbar^2 per row (atomicAdd)
    int write;                            // quantisation: store the BF16 plane (accurate mode)
    unsigned long long *l1;               // quantisation: sum_h |x| 2^(mu'+57) per row, two 32-bit
                                          // halves (l1[2r] high, l1[2r+1] low; atomicAdd)
    int floor_plane;                      // quantisation, componentwise rule: also store
                                          // floor(2^mu' |x|) in plane 1
};

__device__ __forceinline__ int quant_shift(const unsigned long long *row_max, int r) {
    unsigned long long b = row_max[r];
    return b ? 5 - floor_log2_bits(b) : 0;     // zero row: mu' = 0
}

// Partial sums of one row: sum of xbar^2 (fast mode's Cauchy-Schwarz
// majorant; exact: xbar <= 64, k <= 2^17) and sum of floor(|x| 2^(shift+57))
// in two 32-bit halves: each term is an integer below 2^63 because
// |x| 2^shift < 64, so the halves cannot overflow for k <= 2^17 and the sum
// is exact (independent of the order); it is within k 2^-62 (relative) of
// sum |x| 2^shift, the row's 1-norm for the N rule.
struct RowAcc {
    int ss;
    unsigned long long hi, lo;
};

template <typename T>
__device__ __forceinline__ void add_scaled_abs(RowAcc &acc, T x, int shift) {
    const Split sp = split_bits(x);
    const int sh = sp.e + shift + 57;
    // M 2^(sh - 57) = |x| 2^shift < 64, so M << sh < 2^63 whenever sh >= 0
    const uint64_t v = sh >= 0 ? (sh >= 64 ? 0ull : sp.M << sh) : (-sh >= 64 ? 0ull : sp.M >> -sh);
    acc.hi += v >> 32;
    acc.lo += v & 0xFFFFFFFFull;
}

// The row sums of a warp's lanes `mask`-reduced (xor distances < width) and
// added into the row's counters by the lane with (lane & (width-1)) == 0.
__device__ __forceinline__ void flush_row(const PlaneArgs &a, RowAcc acc, int r, int width, bool live) {
    for (int o = 1; o < width; o <<= 1) {
        acc.ss += __shfl_xor_sync(0xffffffffu, acc.ss, o);
        acc.hi += __shfl_xor_sync(0xffffffffu, acc.hi, o);
        acc.lo += __shfl_xor_sync(0xffffffffu, acc.lo, o);
    }
    if (live && (threadIdx.x & (width - 1)) == 0) {
        if (a.sumsq && acc.ss) atomicAdd(a.sumsq + r, acc.ss);
        if (acc.hi) atomicAdd(a.l1 + 2 * r, acc.hi);
        if (acc.lo) atomicAdd(a.l1 + 2 * r + 1, acc.lo);
    }
}

// One element of the quantisation from the bits of x: q = ceil(2^shift |x|)
// and the 1-norm term v = floor(|x| 2^(shift+57)) as 32-bit halves (vhi, vlo).
// A normal double takes one 64-bit shift: |x| 2^shift = M 2^-r < 64 with the
// 53-bit significand M >= 2^52 puts r >= 47, so v = M 2^(57-r) is M shifted
// left by at most 10 (no bit lost: floor(2^shift |x|) = v >> 57 and q adds
// one when any of v's low 57 bits is set) or shifted right (then 2^shift |x|
// < 1/32, so q = 1).  A normal float likewise, with its 24-bit significand
// (r >= 18, a left shift by at most 39).  Zeros and subnormals take the
// general path (ceil_scaled_abs, add_scaled_abs).
template <typename T>
__device__ __forceinline__ void quant_elem(T x, int shift, uint32_t &q, uint32_t &qf, uint32_t &vhi, uint32_t &vlo) {
    if constexpr (sizeof(T) == 8) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        const int ex = int((b >> 52) & 0x7FFu);
        const int r = 1075 - ex - shift;
        if (ex != 0 && ex != 0x7FF && r >= 47) {
            const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
            const int s = 57 - r;                               // <= 10
            const unsigned long long v = (M << max(s, 0)) >> min(max(-s, 0), 63);
            vhi = uint32_t(v >> 32);
            vlo = uint32_t(v);
            qf = vhi >> 25;
            q = s < 0 ? 1u : qf + ((v << 7) != 0ull ? 1u : 0u);
            return;
        }
    } else {
        // FP32: the 24-bit significand M with |x| 2^shift = M 2^-r < 64, r >= 18,
        // so v = M 2^(57-r) is a left shift by at most 39 or a right shift
        const uint32_t b = __float_as_uint(float(x));
        const int ex = int((b >> 23) & 0xFFu);
        const int r = 150 - ex - shift;
        if (ex != 0 && ex != 0xFF && r >= 18) {
            const unsigned long long M = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
            const int s = 57 - r;                               // <= 39
            const unsigned long long v = (M << max(s, 0)) >> min(max(-s, 0), 63);
            vhi = uint32_t(v >> 32);
            vlo = uint32_t(v);
            qf = vhi >> 25;
            q = s < 0 ? 1u : qf + ((v << 7) != 0ull ? 1u : 0u);
            return;
        }
    }
    q = ceil_scaled_abs(x, shift);
    qf = floor_scaled_abs(x, shift);
    RowAcc t{0, 0, 0};
    add_scaled_abs(t, x, shift);
    vhi = uint32_t(t.hi);
    vlo = uint32_t(t.lo);
}

// BF16 of two integers in [0, 127] (exact): the FP32 value of 2^23 + q minus
// 2^23 is q, and its top 16 bits are the BF16 encoding.
__device__ __forceinline__ uint32_t pack_bf16x2_small(uint32_t a, uint32_t b) {
    const float fa = __fsub_rn(__uint_as_float(0x4B000000u | a), 8388608.0f);
    const float fb = __fsub_rn(__uint_as_float(0x4B000000u | b), 8388608.0f);
    return __byte_perm(__float_as_uint(fa), __float_as_uint(fb), 0x7632);
}

// Stores 8 values of Abar (accurate mode), and of floor(2^mu' |x|) in plane 1
// under the componentwise rule, and adds to the row sums.
template <typename T>
__device__ __forceinline__ void emit_quant8(const PlaneArgs &a, const T (&x)[8], int shift, int r, int h0,
                                            RowAcc &acc) {
    uint32_t q[8], qf[8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
        uint32_t vh, vl;
        quant_elem(x[e], shift, q[e], qf[e], vh, vl);
        acc.hi += vh;
        acc.lo += vl;
    }
    if (a.sumsq) {                          // fast mode only
#pragma unroll
        for (int e = 0; e < 8; e++) acc.ss += int(q[e] * q[e]);
    }
    if (a.write) {
        uint4 v;
        v.x = pack_bf16x2_small(q[0], q[1]);
        v.y = pack_bf16x2_small(q[2], q[3]);
        v.z = pack_bf16x2_small(q[4], q[5]);
        v.w = pack_bf16x2_small(q[6], q[7]);
        *reinterpret_cast<uint4 *>(a.out + (long)r * a.k_pad + h0) = v;
    }
    if (a.floor_plane) {
        uint4 v;
        v.x = pack_bf16x2_small(qf[0], qf[1]);
        v.y = pack_bf16x2_small(qf[2], qf[3]);
        v.z = pack_bf16x2_small(qf[4], qf[5]);
        v.w = pack_bf16x2_small(qf[6], qf[7]);
        *reinterpret_cast<uint4 *>(a.out + a.plane + (long)r * a.k_pad + h0) = v;
    }
}

template <typename T>
__device__ __forceinline__ PlaneArgs quant_args(const JobDesc<T> &j, int X) {
    return PlaneArgs{j.res[X], j.plane[X], j.R_pad[X], j.k, j.k_pad, j.rmax[X], nullptr, nullptr,
                     j.fast ? j.ss[X] : nullptr, !j.fast, j.l1[X], j.cw};
}

// Eight consecutive elements src[0 .. 7] of a row, zero from index `valid` on:
// 16-byte vector loads when all eight are in range and src is 16-byte aligned.
__device__ __forceinline__ void load8(const double *src, int valid, double (&x)[8]) {
    if (valid >= 8 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const double2 *v = reinterpret_cast<const double2 *>(src);
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const double2 t = __ldg(v + e);
            x[2 * e] = t.x;
            x[2 * e + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; e++) x[e] = e < valid ? src[e] : 0.0;
    }
}
__device__ __forceinline__ void load8(const float *src, int valid, float (&x)[8]) {
    if (valid >= 8 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const float4 *v = reinterpret_cast<const float4 *>(src);
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const float4 t = __ldg(v + e);
            x[4 * e] = t.x;
            x[4 * e + 1] = t.y;
            x[4 * e + 2] = t.z;
            x[4 * e + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; e++) x[e] = e < valid ? src[e] : 0.0f;
    }
}

// K-contiguous source.  Item: 256 / tpr rows of tpr x 8 h (8 per thread, tpr
// threads per row; each warp lies in one row).  Every lane stays to the end of
// the item (the row sums are reduced across the warp).
template <typename T>
__device__ __forceinline__ void quant_kc_item(const JobDesc<T> &j, long long li) {
    int X = 0;
    const long long n0 = items_quant_kc_x(j, 0);
    if (li >= n0) { X = 1; li -= n0; }
    const PlaneArgs a = quant_args(j, X);
    const Operand<T> &op = j.op[X];
    const int tpr = quant_tpr(a.k_pad), ly = threadIdx.x / tpr, tx = threadIdx.x - ly * tpr;
    const unsigned nhb = unsigned(cdiv(a.k_pad, tpr * 8 * kQuantGroups)), ui = unsigned(li);
    const int rb = int(ui / nhb);
    const int r = rb * (256 / tpr) + ly;
    const int hb = int(ui - unsigned(rb) * nhb) * tpr * 8 * kQuantGroups + tx * 8;
    if (ly >= 256 / tpr) return;            // 256 % tpr threads left over (whole warps)
    RowAcc acc{0, 0, 0};
    const bool live = r < op.R;
    const int shift = live ? quant_shift(a.row_max, r) : 0;
#pragma unroll 2
    for (int g = 0; g < kQuantGroups; g++) {
        const int h0 = hb + g * tpr * 8;    // each chunk coalesced across the row's threads
        if (h0 >= a.k_pad) break;
        if (!live) {
            if (a.write) *reinterpret_cast<uint4 *>(a.out + (long)r * a.k_pad + h0) = make_uint4(0, 0, 0, 0);
            if (a.floor_plane)
                *reinterpret_cast<uint4 *>(a.out + a.plane + (long)r * a.k_pad + h0) = make_uint4(0, 0, 0, 0);
            continue;
        }
        T x[8];
        load8(op.ptr + (long)r * op.ld + h0, a.k - h0, x);
        emit_quant8(a, x, shift, r, h0, acc);
    }
    flush_row(a, acc, r, tpr < 32 ? tpr : 32, live);   // a row's lanes: tpr of them, or whole warps
}

// R-contiguous source.  Item: a 64 (h) x 64 (r) tile transposed through
// shared memory.
template <typename T>
__device__ __forceinline__ void quant_rc_item(const JobDesc<T> &j, long long li, T (*tile)[65]) {
    int X = 0;
    const long long n0 = items_quant_rc_x(j, 0);
    if (li >= n0) { X = 1; li -= n0; }
    const PlaneArgs a = quant_args(j, X);
    const Operand<T> &op = j.op[X];
    const unsigned nrb = unsigned(a.R_pad / 64), ui = unsigned(li);
    const int hb = int(ui / nrb);
    const int h_base = hb * 64, r_base = int(ui - unsigned(hb) * nrb) * 64;
    __syncthreads();                     // the previous item's reads of the tile are done
    {
        const int rr = threadIdx.x & 63;
        const int r = r_base + rr;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int hh = (threadIdx.x >> 6) + 4 * i;
            const int h = h_base + hh;
            tile[hh][rr] = (r < op.R && h < a.k) ? op.ptr[(long)h * op.ld + r] : T(0);
        }
    }
    __syncthreads();
    const int rr = threadIdx.x >> 2, hq = threadIdx.x & 3;
    const int r = r_base + rr;
    const bool live = r < op.R;
    const int shift = live ? quant_shift(a.row_max, r) : 0;
    RowAcc acc{0, 0, 0};
#pragma unroll
    for (int g = 0; g < 2; g++) {
        const int hh0 = hq * 16 + g * 8;
        const int h0 = h_base + hh0;
        T x[8];
#pragma unroll
        for (int e = 0; e < 8; e++) x[e] = live ? tile[hh0 + e][rr] : T(0);
        emit_quant8(a, x, shift, r, h0, acc);
    }
    flush_row(a, acc, r, 4, live);   // the 4 threads of row rr are adjacent lanes
}

// Quantisation of K-contiguous rows.
template <typename T, int CAP>
__global__ void __launch_bounds__(256) k_quant_kc(const __grid_constant__ JobGroup<T, CAP> G) {
    for_items(G, [&](const JobDesc<T> &j, long long li) { quant_kc_item(j, li); });
}

// Quantisation of transposed rows.
template <typename T, int CAP>
__global__ void __launch_bounds__(256) k_quant_rc(const __grid_constant__ JobGroup<T, CAP> G) {
    __shared__ T tile[64][65];
    for_items(G, [&](const JobDesc<T> &j, long long li) { quant_rc_item(j, li, tile); });
}

// Both layouts in one launch, for launches too small to fill the GPU twice
// over: the K-contiguous items of each problem come first, then the
// transposed ones.
template <typename T, int CAP>
__global__ void __launch_bounds__(256) k_quant(const __grid_constant__ JobGroup<T, CAP> G) {
    __shared__ T tile[64][65];
    for_items(G, [&](const JobDesc<T> &j, long long li) {
        const long long nkc = items_quant_kc_x(j, 0) + items_quant_kc_x(j, 1);
        if (li < nkc) quant_kc_item(j, li);
        else quant_rc_item(j, li - nkc, tile);
    });
}

// ------------------------------------------------------------------ residues
// Two FP32 lanes in one 64-bit register (the paired FP32 instructions of
// sm_100 and later).
namespace f2 {
__device__ __forceinline__ unsigned long long pack(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma(unsigned long long a, unsigned long long b,
                                                  unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// BF16x2 of the two lanes (exact here: integers of magnitude <= 128)
__device__ __forceinline__ uint32_t bf16x2(unsigned long long a) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
}  // namespace f2

// Bit length of max_h |x'_rh| for x' = trunc(2^shift x), from the bits of
// max_h |x_rh|: floor(log2 max) + shift + 1 (0 for a zero row).
__device__ __forceinline__ int row_bits(unsigned long long max_bits, int shift) {
    if (!max_bits) return 0;
    const int b = floor_log2_bits(max_bits) + shift + 1;
    return b < 0 ? 0 : b;
}

// Fixed-position limbs (rows whose |x'| < 2^(13 L), L <= 8): x' is cut into L
// 13-bit limbs at bits 0, 13, 26, ..., each carrying the sign of x'.  For odd
// p_l and balanced weights w_i = 2^(13 i) mod p_l:
//   t = sum_i d_i w_i,  |t| <= 8 (2^13 - 1) 127 < 2^23: exact in FP32 (every
//       product and partial sum is an integer below 2^24);
//   q = RN(t RN(1/p) + 1.5 2^23) - 1.5 2^23 = round(t / p): the fma rounds the
//       exact t RN(1/p), which lies strictly within |t| 2^-24 / p < 1/(2p) of
//       t / p, to an integer, and t / p lies at least 1/(2p) from any
//       half-integer (p odd);
//   r = t - q p, the balanced residue of x'.
// Two elements travel together through paired FP32 instructions.
//
// fixed_limbs2: the limbs of two elements as FP32 pairs, the residues mod 256 as BF16x2.
// Limb u (13 bits) becomes the float 2^23 + u by setting the exponent bits,
// and one paired fma s (2^23 + u) - s 2^23 = s u (exact) applies the sign s.
// W64: |x'| < 2^64 (rows of at most 64 bits), so x' is formed in one 64-bit
// word instead of 128 bits.
template <int L, typename T, bool W64 = false>
__device__ __forceinline__ uint32_t fixed_limbs2(T x0, T x1, int shift, unsigned long long (&dp)[L]) {
    Int v0, v1;
    using W = typename std::conditional<W64, unsigned long long, unsigned __int128>::type;
    W w0, w1;
    if constexpr (W64 && sizeof(T) == 8) {
        // x' = trunc(2^shift |x|) < 2^64 straight from the bits: one shift of the
        // significand (subnormals without the implicit bit, non-finite as zero)
        auto one = [&](T x, Int &v) -> unsigned long long {
            const unsigned long long b = (unsigned long long)__double_as_longlong(double(x));
            const int ex = int((b >> 52) & 0x7FFu);
            const unsigned long long M = ex == 0x7FF ? 0ull : (b & 0xFFFFFFFFFFFFFull) | (ex != 0 ? 1ull << 52 : 0ull);
            const int sh = (ex != 0 ? ex : 1) - 1075 + shift;
            v.neg = (b >> 63) != 0;
            return (M << min(max(sh, 0), 63)) >> min(max(-sh, 0), 63);
        };
        w0 = one(x0, v0);
        w1 = one(x1, v1);
    } else {
        v0 = trunc_scaled(x0, shift);
        v1 = trunc_scaled(x1, shift);
        w0 = v0.M == 0 ? W(0) : (W(v0.M) << v0.E);
        w1 = v1.M == 0 ? W(0) : (W(v1.M) << v1.E);
    }
    const unsigned long long sg = f2::pack(v0.neg ? -1.0f : 1.0f, v1.neg ? -1.0f : 1.0f);
    const unsigned long long off = f2::pack(v0.neg ? 8388608.0f : -8388608.0f, v1.neg ? 8388608.0f : -8388608.0f);
#pragma unroll
    for (int i = 0; i < L; i++) {
        const uint32_t a0 = (uint32_t(w0 >> (13 * i)) & 0x1FFFu) | 0x4B000000u;
        const uint32_t a1 = (uint32_t(w1 >> (13 * i)) & 0x1FFFu) | 0x4B000000u;
        dp[i] = f2::fma((unsigned long long)a0 | ((unsigned long long)a1 << 32), sg, off);
    }
    uint32_t b0 = uint32_t(w0) & 255u, b1 = uint32_t(w1) & 255u;
    if (v0.neg) b0 = (256u - b0) & 255u;
    if (v1.neg) b1 = (256u - b1) & 255u;
    return pack_bf16x2f(float(int(int8_t(b0))), float(int(int8_t(b1))));
}

template <int L, typename T, bool W64 = false>
__device__ __forceinline__ void emit_resid8_fixed(uint4 *dst, long pw16, int N, const T (&x)[8], int shift) {
    unsigned long long dp[4][L];
    uint32_t z[4];
#pragma unroll
    for (int j = 0; j < 4; j++) z[j] = fixed_limbs2<L, T, W64>(x[2 * j], x[2 * j + 1], shift, dp[j]);
    dst[0] = make_uint4(z[0], z[1], z[2], z[3]);
    const unsigned long long magic = f2::pack(12582912.0f, 12582912.0f);      // 1.5 2^23
    const unsigned long long nmagic = f2::pack(-12582912.0f, -12582912.0f);
    for (int l = 1; l < N; l++) {
        const unsigned long long *cw = c_w13p[l];
        unsigned long long w[L];
#pragma unroll
        for (int i = 1; i < L; i++) w[i] = cw[i];
        const unsigned long long ip = cw[kFixLimbs], np = cw[kFixLimbs + 1];
        uint32_t o[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            unsigned long long t = dp[j][0];                      // w_0 = 1
#pragma unroll
            for (int i = 1; i < L; i++) t = f2::fma(dp[j][i], w[i], t);
            const unsigned long long q = f2::add(f2::fma(t, ip, magic), nmagic);
            o[j] = f2::bf16x2(f2::fma(q, np, t));
        }
        dst[(long)l * pw16] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// Rows with |x'| >= 2^104: per element, limbs of the mantissa and a second
// reduction by 2^E mod p (residue_odd).
template <typename T>
__device__ __forceinline__ void emit_resid8_general(uint4 *dst, long pw16, int N, const T (&x)[8], int shift,
                                                    const uint8_t (*pow2)[256]) {
    Limbs Lb[8];
#pragma unroll
    for (int e = 0; e < 8; e++) Lb[e] = limbs_of(x[e], shift);
    dst[0] = make_uint4(pack_bf16x2f(float(Lb[0].r256), float(Lb[1].r256)),
                        pack_bf16x2f(float(Lb[2].r256), float(Lb[3].r256)),
                        pack_bf16x2f(float(Lb[4].r256), float(Lb[5].r256)),
                        pack_bf16x2f(float(Lb[6].r256), float(Lb[7].r256)));
    for (int l = 1; l < N; l++) {
        uint32_t o[4];
#pragma unroll
        for (int j = 0; j < 4; j++)
            o[j] = pack_bf16x2f(residue_odd(Lb[2 * j], l, pow2), residue_odd(Lb[2 * j + 1], l, pow2));
        dst[(long)l * pw16] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// Eight consecutive elements of one row; `need` >= the bit length of every |x'|
// of the row (a larger bound only takes more limbs, never a wrong residue).
template <typename T>
__device__ __forceinline__ void emit_resid8(uint4 *dst, long pw16, int N, const T (&x)[8], int shift, int need,
                                            const uint8_t (*pow2)[256]) {
    if (need <= 64) emit_resid8_fixed<5, T, true>(dst, pw16, N, x, shift);
    else if (need <= 65) emit_resid8_fixed<5>(dst, pw16, N, x, shift);
    else if (need <= 78) emit_resid8_fixed<6>(dst, pw16, N, x, shift);
    else if (need <= 104) emit_resid8_fixed<8>(dst, pw16, N, x, shift);
    else emit_resid8_general(dst, pw16, N, x, shift, pow2);
}

__device__ __forceinline__ int warp_max(int v) { return __reduce_max_sync(0xffffffffu, v); }

template <typename T>
__device__ __forceinline__ PlaneArgs resid_args(const JobDesc<T> &j, int X) {
    // the row maxima bound |A'|, |B'| (fixed-position limbs); they are not
    // computed when mu and nu are given
    return PlaneArgs{j.res[X], j.plane[X], j.R_pad[X], j.k, j.k_pad, j.inject ? nullptr : j.rmax[X],
                     j.shift[X], j.ndev, nullptr, 1, nullptr, 0};
}

// K-contiguous source.  Item: 256 consecutive groups of 8 h in row-major order
// (rows shorter than 2048 share an item, so no thread idles); 8 consecutive h
// per thread, one 16-byte store per plane.
template <typename T>
__device__ __forceinline__ void resid_kc_item(const JobDesc<T> &j, long long li, const uint8_t (*pow2)[256]) {
    int X = 0;
    const long long n0 = items_kc_x(j, 0);
    if (li >= n0) { X = 1; li -= n0; }
    const PlaneArgs a = resid_args(j, X);
    const Operand<T> &op = j.op[X];
    const int N = *a.n_dev;
    const long pw16 = a.plane / 8;
    const unsigned k8 = unsigned(a.k_pad / 8);
    const unsigned long long g = (unsigned long long)li * 256u + threadIdx.x;
    const unsigned long long rq = (g >> 32) == 0 ? unsigned(g) / k8 : g / k8;
    if (rq >= (unsigned long long)op.R) return;      // the last item's tail
    const int r = int(rq), h0 = int(g - rq * k8) * 8;
    uint4 *dst = reinterpret_cast<uint4 *>(a.out + (long)r * a.k_pad + h0);
    const int shift = a.shift[r];
    // this row's own bound: where a warp spans several short rows, lanes on
    // both sides of a limb-count limit diverge (rare: the scaling gives
    // neighbouring rows nearly the same bit length; a warp-wide maximum
    // measured slower)
    const int need = a.row_max ? row_bits(a.row_max[r], shift) : 1 << 20;
    T x[8];
    load8(op.ptr + (long)r * op.ld + h0, a.k - h0, x);
    emit_resid8(dst, pw16, N, x, shift, need, pow2);
}

// R-contiguous source, blocks of 128 threads.  Item: a 16 (r) x 128 (h) tile
// transposed through shared memory (rows of 129 doubles), so that each row of
// a plane is written in runs of 256 bytes.  Thread (row rr, group tc < 16) then
// takes h = 8 tc .. 8 tc + 7 of rows rr and rr + 8; within each group of eight
// the elements are stored XOR-permuted by (tc >> 1) & 7, so that the 16 lanes
// of a half-warp reading element e of their groups hit distinct banks (as do
// the 16 rows written per h in the transposing stores).  The last tile of a row may reach past k_pad
// (k_pad is a multiple of 64): those groups are not stored.
__device__ __forceinline__ int resid_swz(int hh) { return hh ^ ((hh >> 4) & 7); }

template <typename T>
__device__ __forceinline__ void resid_rc_item(const JobDesc<T> &j, long long li, const uint8_t (*pow2)[256],
                                              T (*tile)[129]) {
    int X = 0;
    const long long n0 = items_rc_x(j, 0);
    if (li >= n0) { X = 1; li -= n0; }
    const PlaneArgs a = resid_args(j, X);
    const Operand<T> &op = j.op[X];
    const int N = *a.n_dev;
    const long pw16 = a.plane / 8;
    const unsigned nrb = unsigned(cdiv(op.R, 16)), ui = unsigned(li);
    const int hb = int(ui / nrb);
    const int h_base = hb * 128, r_base = int(ui - unsigned(hb) * nrb) * 16;
    __syncthreads();                     // the previous item's reads of the tile are done
    {
        const int rr = threadIdx.x & 15;
        const int r = r_base + rr;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int hh = (threadIdx.x >> 4) + 8 * i;
            const int h = h_base + hh;
            tile[rr][resid_swz(hh)] = (r < op.R && h < a.k) ? op.ptr[(long)h * op.ld + r] : T(0);
        }
    }
    __syncthreads();
    const int tc = threadIdx.x & 15;
    const int h0 = h_base + 8 * tc;
#pragma unroll 1
    for (int i = 0; i < 2; i++) {
        const int rr = (threadIdx.x >> 4) + 8 * i;
        const int r = r_base + rr;
        const bool live = r < op.R;
        const int shift = live ? a.shift[r] : 0;
        const int need = warp_max(live ? (a.row_max ? row_bits(a.row_max[r], shift) : 1 << 20) : 0);
        uint4 *dst = reinterpret_cast<uint4 *>(a.out + (long)r * a.k_pad + h0);
        if (!live || h0 >= a.k_pad) continue;
        T x[8];
#pragma unroll
        for (int e = 0; e < 8; e++) x[e] = tile[rr][resid_swz(8 * tc + e)];
        emit_resid8(dst, pw16, N, x, shift, need, pow2);
    }
}

// Residues of K-contiguous rows (resident blocks looping over the items).
template <typename T, int CAP>
__global__ void __launch_bounds__(256, 3) k_resid_kc(const __grid_constant__ JobGroup<T, CAP> G) {
    for_items(G, [&](const JobDesc<T> &j, long long li) { resid_kc_item(j, li, g_pow2); });
}

// Residues of transposed rows (resident blocks looping over the items).
template <typename T, int CAP>
__global__ void __launch_bounds__(128, 6) k_resid_rc(const __grid_constant__ JobGroup<T, CAP> G) {
    __shared__ T tile[16][129];              // [r][swizzled h]
    for_items(G, [&](const JobDesc<T> &j, long long li) { resid_rc_item(j, li, g_pow2, tile); });
}

// ============================================================= tcgen05 GEMM
namespace gemm {
constexpr int BM = 128, BK = 64;
constexpr int SEG_KB = 16;                       // 1024 K per FP32-exact segment
constexpr int GROUP_M = 8;                       // raster: 8 row tiles per column sweep
constexpr int kThreads = 320;                    // w0 TMA, w1 MMA, w2..w9 epilogue
constexpr int kMaxGroup = 64;                    // problems per launch (kernel parameter space)
constexpr int kMaxBN = 256;                      // widest tile: the padding of n in the workspace
constexpr uint32_t A_BYTES = BM * BK * 2;
// Tile widths BN = 256 (4 stages) and 128 (6 stages) of the same kernel.
template <int BN>
struct Cfg {
    static_assert(BN == 256 || BN == 128, "tile width");
    static constexpr int STAGES = BN == 256 ? 4 : 6;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
    static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t kSmemBytes = STAGES * STAGE_BYTES + 1024 + 256;
    static constexpr uint32_t IDESC = ptx::idesc_bf16_f32<BM, BN>();
    static constexpr int NC = BN / 2;            // columns per epilogue thread
};
}  // namespace gemm

enum { EPI_MAX = 0, EPI_MOD = 1, EPI_CW = 2 };

// One GEMM problem of a launch: X_l (rows l*m_pad ..) times Y_l^T for the planes
// l < planes (and l < *n_dev when n_dev is set), 128 x BN output tiles.
struct GemmProblem {
    CUtensorMap tmA, tmB;      // BF16, K-major, 128B-swizzled boxes of 64 x 128 / 64 x BN
    int m_pad, n_pad, kb_total;
    int tiles_m, tiles_n, planes;
    int plane0;                // first plane of the operands (EPI_CW: plane 1)
    long long item_begin;      // first work item of this problem in the launch
    const int *n_dev;          // EPI_MOD: planes l >= *n_dev are skipped
    int8_t *W;                 // EPI_MOD: W[l*w_plane + row*n_pad + col]
    long long w_plane;
    int *row_max, *col_max;    // EPI_MAX
    const float *cw_row, *cw_col;   // EPI_CW: (a_i, b_i) per row, (c_j, d_j) per column
    unsigned long long *cw_red;     // EPI_CW: maxima of X / L and Y / L (double bits) at [0], [2]
};

template <int CAP = gemm::kMaxGroup>
struct GemmGroup {
    GemmProblem p[CAP];
    int count;
    long long total_items;
    unsigned long long wait_limit_ns;   // limit of every bounded wait (kWaitLimitNs)
    int hook_kb;                        // test hook, -1 normally: at this k-block of its
                                        // first item each CTA's producer arms the stage
                                        // but loads nothing, so the MMA warp's wait expires
};

struct WorkItem {
    int p, l, tile_m, tile_n;
    bool skip;
};

// Work item g -> (problem, plane, tile).  Planes run in order; inside a plane
// the tiles go column by column through groups of GROUP_M row tiles, so the
// CTAs working at the same time share few A and B panels (L2 reuse).
// A role's position in the item space: the problem of its previous item and
// that problem's plane count N (INT_MAX where all planes run).  A role's items
// increase, so the search for the next item's problem resumes there, and N is
// read once per problem.
struct ItemCursor {
    int p = -1, n = 0;
};
template <int CAP>
__device__ __forceinline__ WorkItem decode_item(const GemmGroup<CAP> &G, long long g, ItemCursor &c) {
    WorkItem w;
    int p = c.p < 0 ? 0 : c.p;
    while (p + 1 < G.count && G.p[p + 1].item_begin <= g) p++;
    const GemmProblem &P = G.p[p];
    if (p != c.p) {
        c.p = p;
        c.n = P.n_dev != nullptr ? *P.n_dev : INT_MAX;
    }
    // a problem's items number below 2^31 (tiles x planes), so 32-bit division
    const unsigned li = unsigned(g - P.item_begin);
    const unsigned per_plane = unsigned(P.tiles_m * P.tiles_n);
    w.p = p;
    w.l = int(li / per_plane);
    const unsigned t = li - unsigned(w.l) * per_plane;
    const unsigned span = unsigned(gemm::GROUP_M * P.tiles_n);
    const unsigned grp = t / span;
    const int first_m = int(grp) * gemm::GROUP_M;
    const unsigned gm = unsigned(min(gemm::GROUP_M, P.tiles_m - first_m));
    const unsigned tin = t - grp * span;
    w.tile_m = first_m + int(tin % gm);
    w.tile_n = int(tin / gm);
    w.skip = w.l >= c.n;
    return w;
}

// Planes l >= N come last in a problem's items: a role that meets one moves g
// to the last of its items (g + j gridDim) before the next problem's first, so
// that the loop's increment lands on that first one.
template <int CAP>
__device__ __forceinline__ long long skip_to_next_problem(const GemmGroup<CAP> &G, long long g, int p,
                                                          long long total) {
    const long long next = p + 1 < G.count ? G.p[p + 1].item_begin : total;
    const unsigned steps = (unsigned(next - g) + gridDim.x - 1) / gridDim.x;   // >= 1
    return g + (long long)(steps - 1) * gridDim.x;
}

__device__ __forceinline__ bool bounded_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                             uint64_t limit_ns = kWaitLimitNs) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = ptx::globaltimer();
    while (true) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (ptx::globaltimer() - t0 > limit_ns) {
            *abort_flag = 1;
            atomicOr(&g_status, 1);
            return false;
        }
    }
}

// Every lane waits (each gets the barrier's acquire); the warp proceeds only if
// all lanes saw the phase complete, so .sync.aligned tcgen05 instructions that
// follow are always executed by the whole warp.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          uint64_t limit_ns) {
    const bool ok = bounded_wait(bar, parity, abort_flag, limit_ns);
    return __all_sync(0xffffffffu, ok) != 0;
}

// Teardown after an abort: waits, up to limit_ns and whatever the abort flag
// says, for the phase `parity` of `bar` (the completion of copies or MMAs that
// were already issued), so that the CTA releases its shared memory and TMEM
// only once nothing in flight writes to them.  Gives up with bit 1 of the
// status word set.
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(bar, parity)) {
        if (ptx::globaltimer() - t0 > limit_ns) {
            atomicOr(&g_status, 2);
            return;
        }
    }
}

// 1.5 2^23 in both FP32 lanes, and its negative: x + 1.5 2^23 - 1.5 2^23 rounds
// x to an integer for |x| < 2^22, and the low byte of the bits of r + 1.5 2^23
// is r mod 256 for an integer |r| <= 256
constexpr unsigned long long kMagic2 = 0x4B4000004B400000ull;
constexpr unsigned long long kNegMagic2 = 0xCB400000CB400000ull;

// EPI_MOD, per segment: x, an FP32 accumulator value (an integer, |x| <= 2^24),
// becomes x - p q with q = rint(x RN(1/p)), a representative of x mod p_l with
// |x - p q| <= p/2 + 1 (the FP32 quotient is within 1/2 + 1/p of x / p), two
// elements per paired instruction; these add up exactly in FP32 over the <= 128
// segments of a tile.
__device__ __forceinline__ unsigned long long mod_rep2(unsigned long long x, unsigned long long ip,
                                                        unsigned long long np) {
    const unsigned long long q = f2::add(f2::fma(x, ip, kMagic2), kNegMagic2);
    return f2::fma(q, np, x);
}

// EPI_MOD epilogue of one output tile for one epilogue thread: the NC sums of
// segment representatives (|s| < 2^15) of row `row`, columns col0 .. col0+NC-1,
// reduced to the balanced residue W_l = mod(C'_l, p_l) (exact: |s| < 2^23, and
// s / p lies at least 1/(2p) from a half-integer for odd p; for p = 256 both
// +-128 give the byte 0x80, the class -128) and stored as bytes.
template <int NC>
__device__ __forceinline__ void tile_epilogue_mod(const GemmProblem &P, int l, int row, int col0,
                                                  const unsigned long long (&acc2)[NC / 2]) {
    int8_t *dst = P.W + (long long)l * P.w_plane + (long long)row * P.n_pad + col0;
    const unsigned long long ip = c_w13p[l][kFixLimbs], np = c_w13p[l][kFixLimbs + 1];
#pragma unroll
    for (int g = 0; g < NC / 16; g++) {
        uint32_t w4[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            uint32_t b[4];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const unsigned long long t = f2::add(mod_rep2(acc2[g * 8 + j * 2 + h], ip, np), kMagic2);
                b[2 * h] = uint32_t(t);
                b[2 * h + 1] = uint32_t(t >> 32);
            }
            // the low bytes of four elements, in column order
            w4[j] = __byte_perm(__byte_perm(b[0], b[1], 0x0040), __byte_perm(b[2], b[3], 0x0040), 0x5410);
        }
        *reinterpret_cast<uint4 *>(dst + g * 16) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
}

// EPI_MAX epilogue of one output tile for one epilogue thread: NC INT32 sums of
// row `row`, columns col0 .. col0+NC-1, merged into the row and column maxima.
template <int NC>
__device__ __forceinline__ void tile_epilogue_max(const GemmProblem &P, int row, int col0, int lane,
                                                  const int (&acc)[NC]) {
    {
        int rm = 0;
#pragma unroll
        for (int i = 0; i < NC; i++) rm = max(rm, acc[i]);
        atomicMax(P.row_max + row, rm);
        int mine[NC / 32];
#pragma unroll
        for (int j = 0; j < NC / 32; j++) mine[j] = 0;
#pragma unroll
        for (int c = 0; c < NC; c++) {
            const int v = __reduce_max_sync(0xffffffffu, acc[c]);
            if (lane == (c & 31)) mine[c >> 5] = v;
        }
#pragma unroll
        for (int j = 0; j < NC / 32; j++) atomicMax(P.col_max + col0 + j * 32 + lane, mine[j]);
    }
}

// EPI_CW epilogue (componentwise N rule): Chat_ij = (floor(2^mu' |A|) floor(|B| 2^nu'))_ij
// as INT32 sums; L_ij = 2^-(mu'_i + nu'_j) Chat_ij <= (|A||B|)_ij.  With
// (a, b) = (R_i, 2^alpha'_i) 2^mu'_i and (c, d) = (2^beta'_j, K_j) 2^nu'_j,
//   X_ij / L_ij = (a c + b d) / Chat_ij,   Y_ij / L_ij = b c / Chat_ij,
// the factors of t and t^2 in the N-dependent part of eq. thm:err-1 over L_ij,
// rounded up; an entry with X or Y > 0 and Chat_ij = 0 gives +inf.  Their
// maxima over the thread's entries, then the warp's, go to cw_red.
template <int NC>
__device__ __forceinline__ void tile_epilogue_cw(const GemmProblem &P, int row, int col0, const int (&acc)[NC]) {
    const float2 ab = reinterpret_cast<const float2 *>(P.cw_row)[row];
    const float2 *cd = reinterpret_cast<const float2 *>(P.cw_col) + col0;
    float xm = 0.0f, ym = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; c++) {
        const float2 v = cd[c];
        const float X = __fadd_ru(__fmul_ru(ab.x, v.x), __fmul_ru(ab.y, v.y));
        const float Y = __fmul_ru(ab.y, v.x);
        if (X > 0.0f || Y > 0.0f) {
            if (acc[c] == 0) {
                xm = ym = __int_as_float(0x7f800000);
            } else {
                const float rc = __frcp_ru(__int2float_rd(acc[c]));
                xm = fmaxf(xm, __fmul_ru(X, rc));
                ym = fmaxf(ym, __fmul_ru(Y, rc));
            }
        }
    }
    const unsigned long long bx = warp_max_u64((unsigned long long)__double_as_longlong(double(xm)));
    const unsigned long long by = warp_max_u64((unsigned long long)__double_as_longlong(double(ym)));
    if ((threadIdx.x & 31) == 0) {
        if (bx) atomicMax(P.cw_red, bx);
        if (by) atomicMax(P.cw_red + 2, by);
    }
}

// Persistent CTA (one per SM) working through the items g = blockIdx.x,
// blockIdx.x + gridDim.x, ... of one or more problems.  Each item is a 128 x BN
// tile of X_l Y_l^T (BF16, K-major, integer-valued).  K runs in segments of
// <= 1024 elements: each segment starts a fresh FP32 accumulator in TMEM, so
// every partial sum is an integer of magnitude <= 1024 * 2^14 = 2^24 and exact;
// the epilogue warps turn each segment into INT32 and add it up.  The shared
// memory stage ring and the two TMEM accumulators run on across items, so the
// epilogue of one tile overlaps the MMAs of the next.
//
// Failure path: every wait gives up after G.wait_limit_ns, sets the CTA's abort
// flag (which stops the other roles' loops) and the device status word.  Before
// the CTA frees its TMEM and exits, the producer waits for the loads it issued
// and the MMA warp for the MMAs it issued (drain_wait, bounded again).
template <int EPI, int BN, int CAP>
__global__ void __launch_bounds__(gemm::kThreads, 1) k_gemm(const __grid_constant__ GemmGroup<CAP> G) {
    using namespace gemm;
    using C = Cfg<BN>;
    constexpr int STAGES = C::STAGES;
    constexpr uint32_t STAGE_BYTES = C::STAGE_BYTES, IDESC = C::IDESC;
    constexpr int NC = C::NC;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = ptx::smem_addr(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t *smem = smem_raw + pad;
    const uint32_t sbase = raw + pad;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    auto bar_full = [&](int s) { return ptx::smem_addr(bars + s); };
    auto bar_empty = [&](int s) { return ptx::smem_addr(bars + STAGES + s); };
    auto bar_accf = [&](int b) { return ptx::smem_addr(bars + 2 * STAGES + b); };
    auto bar_acce = [&](int b) { return ptx::smem_addr(bars + 2 * STAGES + 2 + b); };
    const uint32_t bar_drain = ptx::smem_addr(bars + 2 * STAGES + 4);   // MMA teardown after an abort
    const uint64_t limit = G.wait_limit_ns;
    auto sA = [&](int s) { return sbase + uint32_t(s) * STAGE_BYTES; };
    auto sB = [&](int s) { return sbase + uint32_t(s) * STAGE_BYTES + A_BYTES; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) { ptx::mbar_init(bar_full(s), 1); ptx::mbar_init(bar_empty(s), 1); }
        for (int b = 0; b < 2; b++) { ptx::mbar_init(bar_accf(b), 1); ptx::mbar_init(bar_acce(b), 8); }
        ptx::mbar_init(bar_drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc<2 * BN>(ptx::smem_addr(tmem_slot));
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long total = G.total_items;
    uint32_t issued = 0;                         // producer: stages armed (lane 0 of warp 0)

    if (warp == 0) {
        if (lane == 0) {
            uint32_t kbc = 0;                    // stage ring position, across items
            bool ok = true, first = true;
            ItemCursor cur;
            for (long long g = blockIdx.x; g < total && ok; g += gridDim.x) {
                const WorkItem w = decode_item(G, g, cur);
                if (w.skip) { g = skip_to_next_problem(G, g, w.p, total); continue; }
                const GemmProblem &P = G.p[w.p];
                const int row_a = (P.plane0 + w.l) * P.m_pad + w.tile_m * BM;
                const int row_b = (P.plane0 + w.l) * P.n_pad + w.tile_n * BN;
                for (int kb = 0; kb < P.kb_total; kb++, kbc++) {
                    const int s = int(kbc % STAGES);
                    const uint32_t ph = (kbc / STAGES) & 1u;
                    if (kbc >= STAGES && !bounded_wait(bar_empty(s), ph ^ 1u, abort_flag, limit)) { ok = false; break; }
                    ptx::mbar_arrive_expect_tx(bar_full(s), STAGE_BYTES);
                    if (first && kb == G.hook_kb) continue;      // test hook: armed, never loaded
                    ptx::tma_load_2d(sA(s), &P.tmA, kb * BK, row_a, bar_full(s));
                    ptx::tma_load_2d(sB(s), &P.tmB, kb * BK, row_b, bar_full(s));
                }
                first = false;
            }
            issued = kbc;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t kbc = 0, segc = 0;
            bool ok = true;
            ItemCursor cur;
            for (long long g = blockIdx.x; g < total && ok; g += gridDim.x) {
                const WorkItem w = decode_item(G, g, cur);
                if (w.skip) { g = skip_to_next_problem(G, g, w.p, total); continue; }
                const GemmProblem &P = G.p[w.p];
                const int nseg = (P.kb_total + SEG_KB - 1) / SEG_KB;
                for (int seg = 0; seg < nseg && ok; seg++, segc++) {
                    const int buf = int(segc & 1u);
                    if (segc >= 2 && !bounded_wait(bar_acce(buf), ((segc >> 1) - 1) & 1u, abort_flag, limit)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t d = tmem + uint32_t(buf * BN);
                    const int kb0 = seg * SEG_KB;
                    const int kb1 = min(P.kb_total, kb0 + SEG_KB);
                    for (int kb = kb0; kb < kb1; kb++, kbc++) {
                        const int s = int(kbc % STAGES);
                        const uint32_t ph = (kbc / STAGES) & 1u;
                        if (!bounded_wait(bar_full(s), ph, abort_flag, limit)) { ok = false; break; }
                        ptx::tc_fence_after();
#pragma unroll
                        for (int kk = 0; kk < BK / 16; kk++) {
                            const uint64_t ad = ptx::sdesc_sw128_kmajor(sA(s) + uint32_t(kk * 32));
                            const uint64_t bd = ptx::sdesc_sw128_kmajor(sB(s) + uint32_t(kk * 32));
                            ptx::mma_bf16(d, ad, bd, IDESC, (kb > kb0 || kk > 0) ? 1u : 0u);
                        }
                        ptx::mma_commit(bar_empty(s));
                    }
                    if (ok) ptx::mma_commit(bar_accf(buf));
                }
            }
        }
    } else {
        const int q = warp & 3;                 // TMEM lanes 32q..32q+31 (warp rank mod 4)
        const int half = (warp - 2) >> 2;       // columns [NC half, NC half + NC)
        uint32_t segc = 0;
        bool ok = true;
        ItemCursor cur;
        for (long long g = blockIdx.x; g < total && ok; g += gridDim.x) {
            const WorkItem w = decode_item(G, g, cur);
            if (w.skip) { g = skip_to_next_problem(G, g, w.p, total); continue; }
            const GemmProblem &P = G.p[w.p];
            const int nseg = (P.kb_total + SEG_KB - 1) / SEG_KB;
            // EPI_MAX: INT32 sums of the segments; EPI_MOD: FP32 pairs holding the
            // sum of the segments' representatives mod p_l (mod_rep2)
            int acc[EPI == EPI_MOD ? 1 : NC];
            unsigned long long acc2[EPI == EPI_MOD ? NC / 2 : 1];
            unsigned long long ip = 0, np = 0;
            if constexpr (EPI == EPI_MOD) {
#pragma unroll
                for (int i = 0; i < NC / 2; i++) acc2[i] = 0ull;
                ip = c_w13p[w.l][kFixLimbs];
                np = c_w13p[w.l][kFixLimbs + 1];
            } else {
#pragma unroll
                for (int i = 0; i < NC; i++) acc[i] = 0;
            }
            for (int seg = 0; seg < nseg; seg++, segc++) {
                const int buf = int(segc & 1u);
                if (!warp_wait(bar_accf(buf), (segc >> 1) & 1u, abort_flag, limit)) { ok = false; break; }
                ptx::tc_fence_after();
                const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + uint32_t(buf * BN + half * NC);
                if constexpr (EPI == EPI_MOD) {
#pragma unroll
                    for (int c = 0; c < NC / 16; c++) {
                        uint32_t v[16];
                        ptx::tmem_ld_32x32b_x16(taddr + uint32_t(c * 16), v);
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 8; i++) {
                            const unsigned long long x = (unsigned long long)v[2 * i] |
                                                         ((unsigned long long)v[2 * i + 1] << 32);
                            acc2[c * 8 + i] = f2::add(acc2[c * 8 + i], mod_rep2(x, ip, np));
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < NC / 16; c++) {
                        uint32_t v[16];
                        ptx::tmem_ld_32x32b_x16(taddr + uint32_t(c * 16), v);
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 16; i++) acc[c * 16 + i] += __float2int_rn(__uint_as_float(v[i]));
                    }
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(bar_acce(buf));
            }
            if (!ok) break;
            const int row = w.tile_m * BM + q * 32 + lane, col0 = w.tile_n * BN + half * NC;
            if constexpr (EPI == EPI_MOD) tile_epilogue_mod<NC>(P, w.l, row, col0, acc2);
            else if constexpr (EPI == EPI_MAX) tile_epilogue_max<NC>(P, row, col0, lane, acc);
            else tile_epilogue_cw<NC>(P, row, col0, acc);
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    // every role has left its loop; the abort flag no longer changes
    if (*abort_flag && lane == 0) {
        if (warp == 0) {
            // the last STAGES stages armed: their loads (if issued) must land
            for (uint32_t j = issued > uint32_t(STAGES) ? issued - STAGES : 0u; j < issued; j++)
                drain_wait(bar_full(int(j % STAGES)), (j / STAGES) & 1u, limit);
        } else if (warp == 1) {
            // arrives once every MMA this thread issued has completed
            ptx::mma_commit(bar_drain);
            drain_wait(bar_drain, 0, limit);
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc<2 * BN>(tmem);
    }
}

// ============================================================= exponents and N
// red[] holds bits of nonnegative doubles (order-independent atomicMax):
// 0 max_i |A|v, 1 max_j v^T|B|, 2 max_i 2^alpha'_i, 3 max_j 2^beta'_j, 4 L;
// 5 and 7 the componentwise rule's max X / L and max Y / L;
// red[6] as two ints: fast mode's max_i ssA_i, max_j ssB_j.

__device__ __forceinline__ double pow2_prime(unsigned long long rmax_bits, int cmax) {
    // 2^alpha' = 2^alpha sqrt(max cbar) (Theorem 2); 0 for an empty row
    if (rmax_bits == 0 || cmax <= 0) return 0.0;
    return ldexp(sqrt(double(cmax)), floor_log2_bits(rmax_bits)) * (1.0 + 0x1p-40);
}

__device__ __forceinline__ void block_max_to(unsigned long long v, unsigned long long *dst) {
    v = warp_max_u64(v);
    if ((threadIdx.x & 31) == 0 && v) atomicMax(dst, v);
}

// sum_h |x_rh| from the fixed-point counters of the quantisation kernels
__device__ __forceinline__ double row_l1(const unsigned long long *l1, const unsigned long long *rmax, int r) {
    const double v = double(l1[2 * r]) * 4294967296.0 + double(l1[2 * r + 1]);
    return ldexp(v, -(quant_shift(rmax, r) + 57));
}

// Componentwise rule: the row (X = 0) or column (X = 1) factors of X_ij / L_ij
// and Y_ij / L_ij (tile_epilogue_cw), rounded up: the 1-norm times 2^mu' (the
// fixed-point sum lies within k 2^-62 below it; the factor 1 + 2^-30 covers
// that), and 2^alpha' 2^mu' = 2^5 sqrt(max cbar) (2^alpha' of Theorem 2).
template <typename T>
__device__ __forceinline__ void cw_vectors(const JobDesc<T> &j, int X, int t) {
    const unsigned long long rb = j.rmax[X][t];
    float s = 0.0f, w = 0.0f;
    if (rb) {
        const double l1 = (double(j.l1[X][2 * t]) * 4294967296.0 + double(j.l1[X][2 * t + 1])) * 0x1p-57;
        s = __double2float_ru(l1 * (1.0 + 0x1p-30));
        const int cm = j.cmax[X][t];
        w = cm > 0 ? __double2float_ru(sqrt(double(cm)) * 32.0 * (1.0 + 0x1p-40)) : 0.0f;
    }
    // row of A: (a, b) = (R 2^mu', 2^alpha' 2^mu'); column of B: (c, d) = (2^beta' 2^nu', K 2^nu')
    reinterpret_cast<float2 *>(j.cwv[X])[t] = X == 0 ? make_float2(s, w) : make_float2(w, s);
}

// The maxima that the N rule needs.  Item: 256 consecutive indices (one per
// thread) of each of the ranges i < m, j < n, h < k, so that these short,
// latency-bound reductions spread over many SMs.
template <typename T, int CAP>
__global__ void __launch_bounds__(256) k_bound(const __grid_constant__ JobGroup<T, CAP> G) {
    for_items(G, [&](const JobDesc<T> &j, long long li) {
        unsigned long long mR = 0, mK = 0, m2a = 0, m2b = 0, mL = 0;
        {
            const int t = int(li) * 256 + threadIdx.x;
            if (t < j.m) {
                unsigned long long v = (unsigned long long)__double_as_longlong(row_l1(j.l1[0], j.rmax[0], t));
                mR = v > mR ? v : mR;
                v = (unsigned long long)__double_as_longlong(pow2_prime(j.rmax[0][t], j.cmax[0][t]));
                m2a = v > m2a ? v : m2a;
                if (j.cw) cw_vectors(j, 0, t);
            }
            if (t < j.n) {
                unsigned long long v = (unsigned long long)__double_as_longlong(row_l1(j.l1[1], j.rmax[1], t));
                mK = v > mK ? v : mK;
                v = (unsigned long long)__double_as_longlong(pow2_prime(j.rmax[1][t], j.cmax[1][t]));
                m2b = v > m2b ? v : m2b;
                if (j.cw) cw_vectors(j, 1, t);
            }
            if (t < j.k) {
                const double v = __longlong_as_double((long long)j.hmax[0][t]) *
                                 __longlong_as_double((long long)j.hmax[1][t]);
                const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
                mL = bits > mL ? bits : mL;
            }
        }
        block_max_to(mR, j.red + 0);
        block_max_to(mK, j.red + 1);
        block_max_to(m2a, j.red + 2);
        block_max_to(m2b, j.red + 3);
        block_max_to(mL, j.red + 4);
    });
}

// The N rule: smallest N in [2, nmax] with
//   t_N (maxR max2b + max2a maxK) + (k + gN_N) t_N^2 max2a max2b <= tau * L,
// else nmax.  Called by all lanes of one warp: lane c tests N = base + c for
// 32 candidates at a time, and the lowest passing lane decides.
__device__ __forceinline__ bool n_passes(const unsigned long long *red, int c, int k, double tau, int fp32, int cw) {
    const DevN &d = fp32 ? c_n32[c] : c_n64[c];
    if (cw) {
        // componentwise: t_N max(X / L) + (k + gN_N) t_N^2 max(Y / L) <= tau
        const double xm = __longlong_as_double((long long)red[5]);
        const double ym = __longlong_as_double((long long)red[7]);
        return d.t * xm + (double(k) + d.gN) * d.t * d.t * ym <= tau;
    }
    const double maxR = __longlong_as_double((long long)red[0]);
    const double maxK = __longlong_as_double((long long)red[1]);
    const double m2a = __longlong_as_double((long long)red[2]);
    const double m2b = __longlong_as_double((long long)red[3]);
    const double L = __longlong_as_double((long long)red[4]);
    const double T = d.t * (maxR * m2b + m2a * maxK) + (double(k) + d.gN) * d.t * d.t * m2a * m2b;
    return T <= tau * L;
}
__device__ __forceinline__ int choose_n(const unsigned long long *red, int k, double tau, int nmax, int fp32,
                                        int cw) {
    const int lane = threadIdx.x & 31;
    for (int base = 2; base <= nmax; base += 32) {
        const int c = base + lane;
        const unsigned ok = __ballot_sync(0xffffffffu, c <= nmax && n_passes(red, c, k, tau, fp32, cw));
        if (ok) return base + __ffs(int(ok)) - 1;
    }
    return nmax;
}

// N (fixed, or the rule), then Algorithm 2's mu/nu lines: d = single_up(max
// cbar) (1 for an empty row), e = log2f(d) with CUDA's fast __log2f as in the
// paper, mu = mu' + floor(fl_down(fma(c, e, P'))).  Item: 256 of the m + n
// rows and columns (one per thread); every item of a problem derives the same
// N, and item 0 publishes it.
template <typename T, int CAP>
__global__ void __launch_bounds__(256) k_exponents(const __grid_constant__ JobGroup<T, CAP> G) {
    constexpr int fp32 = sizeof(T) == 4 ? 1 : 0;
    __shared__ int sN;
    for_items(G, [&](const JobDesc<T> &j, long long li) {
        __syncthreads();                     // the previous item has read sN
        if (threadIdx.x < 32) {
            const int N = j.nmoduli > 0 ? j.nmoduli : choose_n(j.red, j.k, j.target, j.nmax, fp32, j.cw);
            if (threadIdx.x == 0) {
                sN = N;
                if (li == 0) {
                    *j.ndev = N;
                    if (j.n_out) *j.n_out = N;
                }
            }
        }
        __syncthreads();
        if (j.inject) return;
        const int N = sN;
        const float Pp = fp32 ? c_n32[N].Pprime : c_n64[N].Pprime;
        const float c = c_cneg;
        {
            const int t = int(li) * 256 + threadIdx.x;
            if (t >= j.m + j.n) return;
            const int X = t < j.m ? 0 : 1;
            const int i = X ? t - j.m : t;
            const unsigned long long bits = j.rmax[X][i];
            const int mp = bits ? 5 - floor_log2_bits(bits) : 0;
            const int cm = j.cmax[X][i];
            const float d = cm > 0 ? __int2float_ru(cm) : 1.0f;
            const float ex = __log2f(d);
            const int v = mp + int(floorf(__fmaf_rd(c, ex, Pp)));
            j.expo[X][i] = v;
            if (j.expo_out[X]) j.expo_out[X][i] = v;
        }
    });
}

// Fast mode (a reading; the paper only names the mode): Cbar is replaced by
// its Cauchy-Schwarz majorant chat_ij = ceil(||Abar_i||_2 ||Bbar_j||_2), whose
// row maxima are ceil(sqrt(ssA_i max_j ssB_j)) and column maxima
// ceil(sqrt(max_i ssA_i ssB_j)).  Lemma 0 only needs Dbar >= Cbar and the
// maxima <= 2^12 k, which the majorant satisfies.
template <typename T, int CAP>
__global__ void __launch_bounds__(256) k_fast_max(const __grid_constant__ JobGroup<T, CAP> G) {
    for_items(G, [&](const JobDesc<T> &j, long long li) {
        int a = 0, b = 0;
        const int base = int(li) * 2048 + threadIdx.x;
        for (int e = 0; e < 8; e++) {
            const int t = base + e * 256;
            if (t < j.m) a = max(a, j.ss[0][t]);
            if (t < j.n) b = max(b, j.ss[1][t]);
        }
        a = __reduce_max_sync(0xffffffffu, a);
        b = __reduce_max_sync(0xffffffffu, b);
        int *mx = reinterpret_cast<int *>(j.red + 6);
        if ((threadIdx.x & 31) == 0) {
            if (a) atomicMax(mx, a);
            if (b) atomicMax(mx + 1, b);
        }
    });
}

__device__ __forceinline__ int ceil_sqrt_u64(unsigned long long x) {
    unsigned long long r = (unsigned long long)sqrt(double(x));
    while (r * r > x) r--;
    while ((r + 1) * (r + 1) <= x) r++;
    return int(r * r == x ? r : r + 1);
}

template <typename T, int CAP>
__global__ void __launch_bounds__(256) k_fast_cmax(const __grid_constant__ JobGroup<T, CAP> G) {
    for_items(G, [&](const JobDesc<T> &j, long long li) {
        const int *mx = reinterpret_cast<const int *>(j.red + 6);
        const unsigned long long mA = (unsigned long long)mx[0], mB = (unsigned long long)mx[1];
        const int base = int(li) * 2048 + threadIdx.x;
        for (int e = 0; e < 8; e++) {
            const int t = base + e * 256;
            if (t >= j.m + j.n) break;
            if (t < j.m) j.cmax[0][t] = ceil_sqrt_u64((unsigned long long)j.ss[0][t] * mB);
            else j.cmax[1][t - j.m] = ceil_sqrt_u64(mA * (unsigned long long)j.ss[1][t - j.m]);
        }
    });
}

// ============================================================= CRT
// Algorithm 3 after the products, then Algorithm 1's inverse scaling:
//   C'(1) = sum_l s_l1 W_l, C'(2) = sum_l s_l2 W_l, each the exact sum rounded
//           once to FP64 (b = 64: C'(1) is exact, Lemma 2; b = 32: s_l2 = 0),
//   Q = rint(P_inv C'(1)),  C'' = fma(-Q, P2, fma(-Q, P1, C'(1)) + C'(2)),
//   C = RN(2^-(mu_i + nu_j) C'')  (b = 32: rounded once to FP32).

// ------------------------------------------------------------------ the epilogue's helpers

// RN(x 2^e) where the result leaves the normal range (a call, so that its FP64
// multiplies stay off the common path)
__device__ __noinline__ double scale_pow2_slow(double x, int e) {
    if (e > 1023) return x * 0x1p1023 * 0x1p1023;                 // overflows to +-inf as ldexp does
    if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
    const double y = x * 0x1p-1022;                               // exact: |x| >= 1
    const int e2 = e + 1022;
    if (e2 < -1022) return copysign(0.0, x);
    return y * __longlong_as_double((long long)(e2 + 1023) << 52);
}

// RN(x 2^e) for an integer-valued x with |x| < 2^400 (an exponent add, on the
// integer units, whenever the result stays normal)
__device__ __forceinline__ double scale_pow2(double x, int e) {
    const long long b = __double_as_longlong(x);
    const bool zero = ((unsigned long long)b << 1) == 0;          // +-0, tested on the integer units
    const int ex = int((b >> 52) & 0x7FF);
    if (zero || (ex + e >= 1 && ex + e <= 2046))
        return zero ? x : __longlong_as_double((long long)((unsigned long long)b + ((unsigned long long)(long long)e << 52)));   // exact
    return scale_pow2_slow(x, e);
}

// RN((hi 2^S + lo) 2^e) as a double, from integer operations only (S = 31 or
// 32).  Requires |hi|, |lo| < 2^61 and a result in the normal range (the tables
// check both for every N).  An exact zero gives +0.
template <int S>
__device__ __forceinline__ double rn_sum(long long hi, long long lo, int e) {
    // written without branches (selects only); every shift amount stays in [0, 63]
    const long long t = hi + (lo >> S);            // value = t 2^S + r, 0 <= r < 2^S
    const unsigned long long r = (unsigned long long)lo & ((1ull << S) - 1);
    const bool neg = t < 0;
    // |value| = T 2^S + R
    const unsigned long long T = neg ? ~(unsigned long long)t + (r == 0 ? 1ull : 0ull) : (unsigned long long)t;
    const unsigned long long R = neg ? ((1ull << S) - r) & ((1ull << S) - 1) : r;
    // X 2^s with the bits below 2^s folded into a sticky bit 0 of X (T < 2^63, so s < S)
    const int bt = 64 - __clzll((long long)T);
    const int s = max(bt - (64 - S), 0);
    const unsigned long long X = (T << (S - s)) | (R >> s) | ((R & ((1ull << s) - 1)) != 0 ? 1ull : 0ull);
    const int bl = 64 - __clzll((long long)X);
    const int sh = max(bl - 53, 0);
    unsigned long long mant = bl <= 53 ? X << min(53 - bl, 63) : X >> sh;
    const unsigned long long rem = X & ((1ull << sh) - 1), half = (1ull << sh) >> 1;
    mant += (sh > 0 && (rem > half || (rem == half && (mant & 1ull)))) ? 1ull : 0ull;
    const int carry = int(mant >> 53);
    mant >>= carry;
    const int ex = bl - 1 + s + e + carry;
    const unsigned long long bits = (neg ? (1ull << 63) : 0ull) | ((unsigned long long)(ex + 1023) << 52) |
                                    (mant & ((1ull << 52) - 1));
    return X == 0 ? 0.0 : __longlong_as_double((long long)bits);
}

// H 2^e as a double for |H| < 2^53 (exact, on the integer units; the result is normal).
__device__ __forceinline__ double exact_i53(long long H, int e) {
    const unsigned long long a = H < 0 ? 0ull - (unsigned long long)H : (unsigned long long)H;
    const int bl = 64 - __clzll((long long)a);                     // <= 53 (0 for H = 0)
    const unsigned long long bits = ((unsigned long long)(bl + 1021 + e) << 52) + (a << (53 - bl));
    return H == 0 ? 0.0 : __longlong_as_double((long long)(bits | (H < 0 ? (1ull << 63) : 0ull)));
}

// rint(x) (round half to even, as FP64 rint) on the integer units: the
// fraction bits are rounded off in place, a carry into the exponent field
// giving the next power of two.
__device__ __forceinline__ double rint_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = int((b >> 52) & 0x7FF);
    const unsigned long long sign = b & (1ull << 63);
    const int f = min(max(1075 - e, 1), 52);                     // fraction bits where 1 <= |x| < 2^52
    const unsigned long long t = (b + ((1ull << (f - 1)) - 1) + ((b >> f) & 1ull)) & ~((1ull << f) - 1);
    // |x| < 1: 0, or 1 above 1/2 (1/2 itself goes to the even 0)
    const unsigned long long small = sign | ((b & ~(1ull << 63)) > 0x3FE0000000000000ull ? 0x3FF0000000000000ull : 0ull);
    return __longlong_as_double((long long)(e >= 1075 ? b : (e < 1023 ? small : t)));   // |x| >= 2^52: x
}

// Q = rint(P_inv C'(1)) in FP64 as Algorithm 3 states it, for C'(1) = H g (a
// call: taken only where the integer estimate cannot decide)
__device__ __noinline__ long long crt_q_fp64(long long H, int eg, double Pinv) {
    return (long long)rint_bits(Pinv * exact_i53(H, eg));
}

// c + a.lo16 b.byte0 + a.hi16 b.byte1 (dp2a.lo) or with b's bytes 2, 3
// (dp2a.hi): unsigned 16-bit pieces of a, signed bytes of b.
__device__ __forceinline__ int dp2a_lo(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp2a.lo.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ int dp2a_hi(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp2a.hi.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// One row i, columns j0 .. j0+3 of one thread; load(l) gives the four W_l
// bytes of those columns (zero for l >= N).  C'(1) and C'(2) are sums of
// integer multiples of fixed grids, taken exactly: each constant is cut into
// 16-bit pieces (s_l1 / g, below 2^48, into three; s_l2 / 2^esum into four),
// and one dp2a adds piece * W for two planes of one column into a 32-bit sum
// (|sum| < 2^16 128 49 < 2^31).  The piece sums are then put
// together in 64-bit integers and rounded once.
template <typename T, int AHEAD, typename Load>
__device__ __forceinline__ void crt_row(const Load &load, int N, const DevN &d, const int32_t *mu,
                                        const int32_t *nu, T *C, long ldc, int n, int i, int j0, bool accum) {
    constexpr int B = sizeof(T) == 8 ? 64 : 32;
    int s1[4][3], s2[4][4];                    // [column][piece]: C'(1) (b = 64 only), C'(2) / b = 32 C'(1)
#pragma unroll
    for (int e = 0; e < 4; e++) {
#pragma unroll
        for (int q = 0; q < 3; q++) s1[e][q] = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) s2[e][q] = 0;
    }
    const int pairs = (N + 1) / 2;
    // software pipeline: the next AHEAD (1 or 2) pairs' loads are in flight while a pair is summed
    static_assert(AHEAD == 1 || AHEAD == 2, "prefetch depth");
    uint32_t w0 = load(0), w1 = load(1), v0 = AHEAD == 2 ? load(2) : 0u, v1 = AHEAD == 2 ? load(3) : 0u;
    for (int pi = 0; pi < pairs; pi++) {
        const uint32_t p0 = w0, p1 = w1;
        if (AHEAD == 2) {
            w0 = v0;
            w1 = v1;
            v0 = load(2 * pi + 4);
            v1 = load(2 * pi + 5);
        } else {
            w0 = load(2 * pi + 2);
            w1 = load(2 * pi + 3);
        }
        // bytes of columns (0, 1) and (2, 3), planes 2 pi and 2 pi + 1 side by side
        const uint32_t x01 = __byte_perm(p0, p1, 0x5140), x23 = __byte_perm(p0, p1, 0x7362);
        const uint4 c2 = B == 64 ? c_dp64[d.poff + pi][1] : c_dp32[d.poff + pi];
        const uint32_t cc2[4] = {c2.x, c2.y, c2.z, c2.w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            s2[0][q] = dp2a_lo(cc2[q], x01, s2[0][q]);
            s2[1][q] = dp2a_hi(cc2[q], x01, s2[1][q]);
            s2[2][q] = dp2a_lo(cc2[q], x23, s2[2][q]);
            s2[3][q] = dp2a_hi(cc2[q], x23, s2[3][q]);
        }
        if (B == 64) {
            const uint4 c1 = c_dp64[d.poff + pi][0];   // piece 3 is zero: s_l1 / g < 2^48
            const uint32_t cc1[3] = {c1.x, c1.y, c1.z};
#pragma unroll
            for (int q = 0; q < 3; q++) {
                s1[0][q] = dp2a_lo(cc1[q], x01, s1[0][q]);
                s1[1][q] = dp2a_hi(cc1[q], x01, s1[1][q]);
                s1[2][q] = dp2a_lo(cc1[q], x23, s1[2][q]);
                s1[3][q] = dp2a_hi(cc1[q], x23, s1[3][q]);
            }
        }
    }
    const int mi = mu[i];
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const int j = j0 + e;
        if (j >= n) break;
        // the second sum as hi 2^32 + lo: pieces 0, 1 and 2, 3 (shifted as unsigned:
        // the sums may be negative)
        const long long lo2 = (long long)((unsigned long long)(long long)s2[e][0] +
                                          ((unsigned long long)(long long)s2[e][1] << 16));
        const long long hi2 = (long long)((unsigned long long)(long long)s2[e][2] +
                                          ((unsigned long long)(long long)s2[e][3] << 16));
        double cpp;
        if (B == 64) {
            // C'(1) = H g exactly, |H| < 2^53 (Lemma 2): the three piece sums added
            // modulo 2^64, which is exact because H fits
            const unsigned long long Hu = (unsigned long long)(long long)s1[e][0] +
                                          ((unsigned long long)(long long)s1[e][1] << 16) +
                                          ((unsigned long long)(long long)s1[e][2] << 32);
            // Q: y = (H >> 22) kq 2^-sq is within 2^-15 of H g / P and FP64's
            // P_inv C'(1) within 2^-38 of it, so both have the nearest integer
            // of y unless y lies within 2^-14 of a half-integer (then FP64 decides)
            const long long H = (long long)Hu;
            const long long z = (long long)(int)(H >> 22) * (long long)d.kq;
            const unsigned long long half = 1ull << (d.sq - 1);
            const unsigned long long fr = (unsigned long long)z & ((half << 1) - 1);
            long long q = (long long)((unsigned long long)z + half) >> d.sq;
            if ((fr > half ? fr - half : half - fr) <= (half >> 13)) q = crt_q_fp64(H, d.eg, d.Pinv);
            // fma(-Q, P1, C'(1)) is exact (|C'(1) - Q P1| < 2^53 ulp(P1), both
            // multiples of ulp(P1) = 2^eu1): T1 2^eu1, taken modulo 2^64
            const long long T1 = (long long)(((unsigned long long)H << d.sh) -
                                             (unsigned long long)q * (unsigned long long)d.M1);
            // C'(2) = RN(hi2 2^32 + lo2) 2^esum as the sum of two exact doubles
            const long long th = hi2 + (lo2 >> 32);
            const long long tl = lo2 & 0xFFFFFFFFll;
            const double c2 = exact_i53(th, d.esum + 32) + exact_i53(tl, d.esum);
            cpp = fma(-exact_i53(q, 0), d.P2, exact_i53(T1, d.eu1) + c2);
        } else {
            const double c1 = rn_sum<32>(hi2, lo2, d.esum);
            const double q = rint_bits(d.Pinv * c1);
            // P2 = 0 and C'(2) = +0, so fma(-q, 0, x + 0) = x + 0 as in the b = 64 form
            cpp = fma(-q, d.P1, c1) + 0.0;
        }
        const double v = scale_pow2(cpp, -(mi + nu[j]));
        const T c = B == 64 ? T(v) : T(__double2float_rn(v));
        T *dst = C + (long)i * ldc + j;
        *dst = accum ? *dst + c : c;            // one rounding per added K range
    }
}

// One problem: block (x, y) takes columns 1024 x .. 1024 x + 1023 of rows y,
// y + gridDim.y, ...
constexpr int kCrtCols = 1024;
template <typename T>
__global__ void __launch_bounds__(256) k_crt_one(const int8_t *W, long w_plane, long n_pad, const int *n_dev,
                                                 const int32_t *mu, const int32_t *nu, T *C, long ldc, int m, int n,
                                                 int accum) {
    const int N = *n_dev;
    const DevN d = sizeof(T) == 8 ? c_n64[N] : c_n32[N];
    const long col0 = (long)blockIdx.x * kCrtCols;
    const int j0 = int(col0) + threadIdx.x * 4;
    for (int i = blockIdx.y; i < m; i += gridDim.y) {
        if (j0 >= n) continue;
        const int8_t *wp = W + (long)i * n_pad + j0;
        crt_row<T, 2>([&](int l) { return l < N ? __ldg(reinterpret_cast<const uint32_t *>(wp + (long)l * w_plane)) : 0u; },
                   N, d, mu, nu, C, ldc, n, i, j0, accum != 0);
    }
}

// A group of problems.  Item: 256 consecutive groups of 4 columns in the
// problem's row-major order (ceil(n / 4) groups per row; rows shorter than 1024
// share an item, so no thread idles), 4 columns per thread.
template <typename T, int CAP>
__global__ void __launch_bounds__(256, 4) k_crt(const __grid_constant__ JobGroup<T, CAP> G) {
    for_items(G, [&](const JobDesc<T> &jd, long long li) {
        const unsigned q = unsigned(cdiv(jd.n, 4));
        const unsigned long long g = (unsigned long long)li * 256u + threadIdx.x;
        const unsigned long long iq = (g >> 32) == 0 ? unsigned(g) / q : g / q;
        if (iq >= (unsigned long long)jd.m) return;            // the last item's tail
        const int i = int(iq), j0 = int(g - iq * q) * 4;
        const int N = *jd.ndev;
        const DevN d = sizeof(T) == 8 ? c_n64[N] : c_n32[N];
        const int8_t *wp = jd.W + (long)i * jd.n_pad + j0;
        const long wpl = jd.w_plane;
        crt_row<T, 2>([&](int l) { return l < N ? __ldg(reinterpret_cast<const uint32_t *>(wp + (long)l * wpl)) : 0u; },
                   N, d, jd.shift[0], jd.shift[1], jd.C, jd.ldc, jd.n, i, j0, jd.accum != 0);
    });
}

// ============================================================= complex operands
// A complex product as two real ones: with A_s = [Re op(A), Im op(A)] (m x 2k),
//   Re C = A_s [Re op(B); -Im op(B)],   Im C = A_s [Im op(B); Re op(B)],
// each one real emulated GEMM over 2k.  k_zsplit copies an interleaved complex
// matrix X (R x L complex, row stride ldx complex) into a real one whose rows
// hold two halves, each the real or the imaginary part of X with a sign:
// side by side (row r = [half 0 of row r, half 1 of row r], R x 2L) or stacked
// (rows r and R + r, 2R x L).  X is 2 sizeof(T)-aligned (checked on the host).
template <typename T>
struct Cplx;
template <>
struct Cplx<double> { using V = double2; };
template <>
struct Cplx<float> { using V = float2; };

template <typename T>
__global__ void __launch_bounds__(256) k_zsplit(const T *X, long ldx, int R, int L, int stacked, int im0, int neg0,
                                                int im1, int neg1, T *Y, long ldy) {
    using V = typename Cplx<T>::V;
    const int c = blockIdx.x * 256 + threadIdx.x;
    if (c >= L) return;
    for (int r = blockIdx.y; r < R; r += gridDim.y) {
        const V x = reinterpret_cast<const V *>(X)[(long)r * ldx + c];
        const T h0 = im0 ? x.y : x.x, h1 = im1 ? x.y : x.x;
        T *row = Y + (long)r * ldy;
        row[c] = neg0 ? -h0 : h0;
        if (stacked) Y[(long)(R + r) * ldy + c] = neg1 ? -h1 : h1;
        else row[L + c] = neg1 ? -h1 : h1;
    }
}

// C (m x n complex, row stride ldc complex) = Re + i Im (both m x n real, ld).
template <typename T>
__global__ void __launch_bounds__(256) k_zmerge(const T *Re, const T *Im, long ld, int m, int n, T *C, long ldc) {
    using V = typename Cplx<T>::V;
    const int j = blockIdx.x * 256 + threadIdx.x;
    if (j >= n) return;
    for (int i = blockIdx.y; i < m; i += gridDim.y) {
        V v;
        v.x = Re[(long)i * ld + j];
        v.y = Im[(long)i * ld + j];
        reinterpret_cast<V *>(C)[(long)i * ldc + j] = v;
    }
}

// ============================================================= diagnostics
// The failure path of the bounded waits, without a fault: one thread waits on
// an mbarrier that nothing arrives on, with the GEMM's wait loop and a limit of
// limit_ns; the wait gives up, sets the device status word (which oz2_sync
// turns into OZ2_ETIMEOUT) and the kernel returns normally.
__global__ void k_wait_selftest(uint64_t limit_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    abort_flag = 0;
    const uint32_t b = ptx::smem_addr(&bar);
    ptx::mbar_init(b, 1);
    ptx::fence_mbar_init();
    bounded_wait(b, 0, &abort_flag, limit_ns);
}

// Assumption (1), Section 1.2: |log2f(x) - log2 x| <= 4 u32 log2 x, checked
// for CUDA's __log2f on every FP32 value x that is an integer in [1, 2^29]
// (the values Dbar can take).  out[0] += violations, out[1] = max ratio
// |err| / (u32 log2 x) as double bits (atomicMax).
__global__ void __launch_bounds__(256) k_log2f_check(uint32_t first_bits, uint32_t count,
                                                     unsigned long long *out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned long long bad = 0, worst = 0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
        const float x = __uint_as_float(first_bits + t);
        if (x != truncf(x)) continue;
        const double lx = log2(double(x));
        const double err = fabs(double(__log2f(x)) - lx);
        if (err > 4.0 * 0x1p-24 * lx) bad++;
        if (lx > 0) {
            const double ratio = err / (0x1p-24 * lx);
            const unsigned long long b = (unsigned long long)__double_as_longlong(ratio);
            worst = b > worst ? b : worst;
        }
    }
    if (bad) atomicAdd(out, bad);
    for (int o = 16; o; o >>= 1) {
        unsigned long long t2 = __shfl_xor_sync(0xffffffffu, worst, o);
        worst = t2 > worst ? t2 : worst;
    }
    if ((threadIdx.x & 31) == 0 && worst) atomicMax(out + 1, worst);
}

}  // namespace oz2
