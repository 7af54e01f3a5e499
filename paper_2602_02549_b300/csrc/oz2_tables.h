// Host-side constant tables of the Ozaki-II scheme, generated at load time
// from the moduli of eq. (p_list) with a small multi-precision integer.
#pragma once
#include <cstdint>

namespace oz2 {

constexpr int kNMax = 49;
constexpr int kLimbs = 5;                               // 12-bit limbs of a 53-bit mantissa
constexpr int kFixLimbs = 8;                            // 13-bit limbs of an integer below 2^104
constexpr int kPackedLen = (kNMax * (kNMax + 1)) / 2;  // sum_{N=1}^{49} N entries
constexpr int kPairsLen = 625;                          // sum_{N=1}^{49} ceil(N / 2) plane pairs

// Per-modulus reduction constants (index l = 0..48).
struct ModTable {
    int p[kNMax];
    uint8_t pow2[kNMax][256];// 2^E mod p, E = 0..255
    float w12[kNMax][kLimbs];     // balanced 2^(12 j) mod p, in [-(p-1)/2, (p-1)/2] (odd p)
    // {w, w} pairs of FP32 bits: balanced 2^(13 j) mod p (j < kFixLimbs), RN(1/p), -p
    unsigned long long w13p[kNMax][kFixLimbs + 2];
    float pf[kNMax];         // p as float
    float invp[kNMax];       // RN_f32(1/p)
};

// Per-N scalars for one precision (b = 64 or 32).
struct NTable {
    double P1, P2, Pinv;     // P1 + P2 ~ P (P2 = 0 for b = 32), Pinv = double(1/P)
    double g;                // grid of s_l1 (b = 64); 1 for b = 32 (unused)
    double t;                // 1/sqrt(32 (P-1)), rounded up
    double gN;               // P-proportional part of R_b (Lemma 4), rounded up
    float Pprime;            // single_down(log2(P-1)/2 - 0.5)
    int offset;              // start of this N's entries in the packed arrays
    int eg;                  // b = 64: g = 2^eg
    int esum;                // grid of the rounded CRT sum: s_l2 (b = 64) or s_l1
                             // (b = 32) = (k[1] 2^31 + k[0]) 2^esum
    int poff;                // start of this N's plane pairs in dp64 / dp32
    // b = 64, the CRT kernel's integer steps: P1 = M1 2^eu1 (M1 < 2^53), g = 2^(eu1 + sh);
    // Q's estimate (H >> 22) kq 2^-sq ~ H g / P for C'(1) = H g
    long long M1;
    int eu1, sh, kq, sq;
};

struct Tables {
    ModTable mod;
    NTable n64[kNMax + 1];
    NTable n32[kNMax + 1];
    long long s1i[kPackedLen];   // b = 64: s_l1 / g, an integer below 2^53
    double s1d[kPackedLen];      // b = 64: s_l1
    double s2d[kPackedLen];      // b = 64: s_l2
    double s1f[kPackedLen];      // b = 32: s_l1 = double(P/p_l q_l)
    // The constants of the two CRT sums as integers on a common grid, split
    // into 31-bit halves (k = k[1] 2^31 + k[0], 0 <= k < 2^62):
    int s1s[kPackedLen][2];      // b = 64: s_l1 / g
    int ks64[kPackedLen][2];     // b = 64: s_l2 / 2^esum
    int ks32[kPackedLen][2];     // b = 32: s_l1 / 2^esum
    // The same constants as 16-bit pieces for the CRT kernel's dp2a sums: for the
    // plane pair (l, l + 1) = (2 i, 2 i + 1) of N, word j holds piece j (bits
    // 16 j .. 16 j + 15) of the constant of plane l in its low half and of plane
    // l + 1 (0 when l + 1 = N) in its high half.
    uint32_t dp64[kPairsLen][8]; // b = 64: words 0-3 pieces of s_l1 / g, 4-7 of s_l2 / 2^esum
    uint32_t dp32[kPairsLen][4]; // b = 32: pieces of s_l1 / 2^esum
    bool sums_fit;               // every k above is below 2^62 and every grid in range
    float c;                     // single_down(-0.5 / (1 - 4 u32))
};

// Built once (thread-safe); never fails for N in [2, 49].
const Tables &tables();

}  // namespace oz2
