// Constant tables of the Ozaki-II scheme (arXiv 2602.02549), computed on the
// host with a minimal unsigned multi-precision integer (P reaches 2^342).
//
//   Theorem 1 / Step 1:  P = prod p_l, q_l = (P/p_l)^-1 mod p_l, q_l < p_l.
//   Section 3.1:         P1 = double(P); P2 = double(P - P1) (b = 64) or 0;
//                        b = 64: s_l1 keeps the upper beta_l bits of P/p_l q_l,
//                        i.e. truncation onto the grid
//                        g = 2^(ceil(log2 rho) + floor(log2 r) - 52),
//                        r = max_l P/p_l q_l, and s_l2 = double(rest);
//                        b = 32: s_l1 = double(P/p_l q_l), s_l2 = 0.
//   Algorithm 2:         P' = single_down(log2(P-1)/2 - 0.5),
//                        c  = single_down(-0.5/(1 - 4 u32)).
//   Algorithm 3:         P_inv = double(1/P).
//   Theorem 2, Lemma 4:  t = 1/sqrt(2^5 (P-1)), the P-proportional part of R_b.
#include "oz2_tables.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

namespace oz2 {
namespace {

// eq. (p_list): the moduli in the order the paper fixes; N uses the first N.
constexpr int kModuli[kNMax] = {
    256, 255, 253, 251, 247, 241, 239, 233, 229, 227,
    223, 217, 211, 199, 197, 193, 191, 181, 179, 173,
    167, 163, 157, 151, 149, 139, 137, 131, 127, 113,
    109, 107, 103, 101, 97,  89,  83,  79,  73,  71,
    67,  61,  59,  53,  47,  43,  41,  37,  29};

// Little-endian base-2^32 unsigned integer, no leading zero limbs.
struct Big {
    std::vector<uint32_t> w;

    static Big of(uint64_t v) {
        Big b;
        while (v) { b.w.push_back(uint32_t(v)); v >>= 32; }
        return b;
    }
    void trim() { while (!w.empty() && w.back() == 0) w.pop_back(); }
    bool zero() const { return w.empty(); }
    int bits() const {
        if (w.empty()) return 0;
        return int(w.size() - 1) * 32 + (32 - __builtin_clz(w.back()));
    }
    bool bit(int i) const {
        size_t li = size_t(i) >> 5;
        return li < w.size() && ((w[li] >> (i & 31)) & 1u);
    }
    Big mul(uint32_t s) const {
        Big r;
        uint64_t carry = 0;
        for (uint32_t x : w) {
            uint64_t t = uint64_t(x) * s + carry;
            r.w.push_back(uint32_t(t));
            carry = t >> 32;
        }
        if (carry) r.w.push_back(uint32_t(carry));
        r.trim();
        return r;
    }
    Big div(uint32_t d, uint32_t *rem) const {
        Big q;
        q.w.assign(w.size(), 0);
        uint64_t r = 0;
        for (size_t i = w.size(); i-- > 0;) {
            uint64_t cur = (r << 32) | w[i];
            q.w[i] = uint32_t(cur / d);
            r = cur % d;
        }
        q.trim();
        if (rem) *rem = uint32_t(r);
        return q;
    }
    Big shr(int s) const {
        Big r;
        int ls = s >> 5, bs = s & 31;
        for (size_t i = size_t(ls); i < w.size(); i++) {
            uint64_t v = w[i] >> bs;
            if (bs && i + 1 < w.size()) v |= uint64_t(w[i + 1]) << (32 - bs);
            r.w.push_back(uint32_t(v));
        }
        r.trim();
        return r;
    }
    Big shl(int s) const {
        Big r;
        int ls = s >> 5, bs = s & 31;
        r.w.assign(size_t(ls), 0);
        uint32_t carry = 0;
        for (uint32_t x : w) {
            r.w.push_back((x << bs) | carry);
            carry = bs ? (x >> (32 - bs)) : 0;
        }
        if (carry) r.w.push_back(carry);
        r.trim();
        return r;
    }
    Big low(int s) const {   // this mod 2^s
        Big r = *this;
        size_t keep = size_t((s + 31) >> 5);
        if (r.w.size() > keep) r.w.resize(keep);
        if ((s & 31) && r.w.size() == keep) r.w[keep - 1] &= (1u << (s & 31)) - 1u;
        r.trim();
        return r;
    }
    uint64_t u64() const {
        uint64_t v = 0;
        for (size_t i = w.size(); i-- > 0;) v = (v << 32) | w[i];
        return v;
    }
};

int cmp(const Big &a, const Big &b) {
    if (a.w.size() != b.w.size()) return a.w.size() < b.w.size() ? -1 : 1;
    for (size_t i = a.w.size(); i-- > 0;)
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
    return 0;
}

Big sub(const Big &a, const Big &b) {   // a >= b
    Big r;
    int64_t borrow = 0;
    for (size_t i = 0; i < a.w.size(); i++) {
        int64_t t = int64_t(a.w[i]) - (i < b.w.size() ? int64_t(b.w[i]) : 0) - borrow;
        borrow = t < 0;
        r.w.push_back(uint32_t(t + (borrow ? (int64_t(1) << 32) : 0)));
    }
    r.trim();
    return r;
}

// Round-to-nearest-even of x * 2^scale2, where `sticky` means the true value
// is strictly greater than x (a nonzero tail below x's last bit).
double round_big(const Big &x, bool sticky, int scale2) {
    int nb = x.bits();
    if (nb == 0) return 0.0;
    if (nb <= 53 && !sticky) return std::ldexp(double(x.u64()), scale2);
    if (nb <= 53) {
        Big y = x.shl(60);   // room for the round and sticky bits
        return round_big(y, true, scale2 - 60);
    }
    int sh = nb - 53;
    uint64_t m = x.shr(sh).u64();
    bool half = x.bit(sh - 1);
    bool rest = sticky || !x.low(sh - 1).zero();
    if (half && (rest || (m & 1))) m++;
    return std::ldexp(double(m), scale2 + sh);
}

double to_double(const Big &x) { return round_big(x, false, 0); }

// double(1/P): long division of 2^s by P, then one rounding.
double reciprocal(const Big &P) {
    int s = P.bits() + 70;
    Big q, r;
    for (int i = s; i >= 0; i--) {
        r = r.shl(1);
        if (i == s) r = Big::of(1);
        q = q.shl(1);
        if (cmp(r, P) >= 0) {
            r = sub(r, P);
            if (q.w.empty()) q = Big::of(1);
            else q.w[0] |= 1u;
        }
    }
    return round_big(q, !r.zero(), -s);
}

long double to_ld(const Big &x) {
    int nb = x.bits();
    if (nb <= 64) return (long double)x.u64();
    return std::ldexp((long double)x.shr(nb - 64).u64(), nb - 64);
}

uint32_t inv_mod(uint32_t a, uint32_t p) {   // a^-1 mod p, gcd(a, p) = 1
    int64_t t = 0, nt = 1, r = p, nr = a % p;
    while (nr) {
        int64_t q = r / nr;
        int64_t tmp = t - q * nt; t = nt; nt = tmp;
        tmp = r - q * nr; r = nr; nr = tmp;
    }
    if (t < 0) t += p;
    return uint32_t(t);
}

float f32_down(long double v) {
    float f = float(v);
    if ((long double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
}

int ceil_log2_u(uint64_t x) { return x <= 1 ? 0 : 64 - __builtin_clzll(x - 1); }

// s_l = k_l 2^e for nonnegative doubles s_0..s_{N-1}: e is the exponent of the
// least significant mantissa bit over all nonzero s_l, so every k_l is an
// integer.  False if some k_l reaches 2^62 (the device sum would overflow) or
// a result grid would leave the normal range.
bool split_on_grid(const double *s, int N, int (*k)[2], int *e_out) {
    int e = INT_MAX;
    for (int l = 0; l < N; l++) {
        if (s[l] == 0.0) continue;
        if (!(s[l] > 0.0)) return false;
        int ex;
        std::frexp(s[l], &ex);
        e = std::min(e, ex - 53);
    }
    if (e == INT_MAX) e = 0;
    *e_out = e;
    bool ok = e >= -1022 && e + 80 <= 1023;
    for (int l = 0; l < N; l++) {
        const double kd = std::ldexp(s[l], -e);
        ok &= kd < 0x1p62;
        const uint64_t v = ok ? uint64_t(kd) : 0;
        k[l][0] = int(v & 0x7FFFFFFFu);
        k[l][1] = int(v >> 31);
    }
    return ok;
}

void build(Tables &T) {
    std::memset(&T, 0, sizeof T);
    for (int l = 0; l < kNMax; l++) {
        uint32_t p = uint32_t(kModuli[l]);
        T.mod.p[l] = int(p);
        uint32_t v = 1 % p;
        for (int e = 0; e < 256; e++) { T.mod.pow2[l][e] = uint8_t(v); v = (v * 2) % p; }
        v = 1 % p;
        for (int j = 0; j < kLimbs; j++) {
            const int bal = 2 * v > p ? int(v) - int(p) : int(v);
            T.mod.w12[l][j] = float(bal);
            v = uint32_t((uint64_t(v) << 12) % p);
        }
        T.mod.pf[l] = float(p);
        T.mod.invp[l] = 1.0f / float(p);
        auto dup = [](float f) {
            uint32_t b;
            std::memcpy(&b, &f, 4);
            return (uint64_t(b) << 32) | b;
        };
        v = 1 % p;
        for (int j = 0; j < kFixLimbs; j++) {
            const int bal = 2 * v > p ? int(v) - int(p) : int(v);
            T.mod.w13p[l][j] = dup(float(bal));
            v = uint32_t((uint64_t(v) << 13) % p);
        }
        T.mod.w13p[l][kFixLimbs] = dup(T.mod.invp[l]);
        T.mod.w13p[l][kFixLimbs + 1] = dup(-float(p));
    }
    const long double u64 = 0x1p-53L, u32 = 0x1p-24L;
    T.c = f32_down(-0.5L / (1.0L - 4.0L * u32));
    int offset = 0, poff = 0;
    T.sums_fit = true;
    for (int N = 1; N <= kNMax; N++) {
        Big P = Big::of(1);
        uint64_t rho = 0;
        for (int l = 0; l < N; l++) { P = P.mul(uint32_t(kModuli[l])); rho += uint64_t(kModuli[l] / 2); }
        std::vector<Big> x;
        x.resize(size_t(N));
        Big r;
        for (int l = 0; l < N; l++) {
            uint32_t p = uint32_t(kModuli[l]), rem = 0;
            Big Pp = P.div(p, nullptr);
            Pp.div(p, &rem);
            uint32_t q = inv_mod(rem, p);
            x[size_t(l)] = Pp.mul(q);
            if (cmp(x[size_t(l)], r) > 0) r = x[size_t(l)];
        }
        const Big Pm1 = sub(P, Big::of(1));
        const int nb = Pm1.bits();
        long double lg = (long double)(nb > 64 ? nb - 64 : 0) +
                         std::log2((long double)(nb > 64 ? Pm1.shr(nb - 64).u64() : Pm1.u64()));
        const float Pprime = f32_down(lg / 2.0L - 0.5L);
        const double P1 = to_double(P);
        const double Pinv = reciprocal(P);
        const long double PL = to_ld(P);
        const double t = double(1.0L / std::sqrt(32.0L * to_ld(Pm1))) * (1.0 + 0x1p-45);
        const int clr = ceil_log2_u(rho);

        {   // b = 64
            NTable &n = T.n64[N];
            n.P1 = P1;
            int e1;
            double f1 = std::frexp(P1, &e1);
            Big P1b = Big::of(uint64_t(std::ldexp(f1, 53)));
            P1b = e1 - 53 >= 0 ? P1b.shl(e1 - 53) : P1b.shr(53 - e1);
            n.P2 = cmp(P, P1b) >= 0 ? to_double(sub(P, P1b)) : -to_double(sub(P1b, P));
            n.Pinv = Pinv;
            n.M1 = (long long)std::ldexp(f1, 53);
            n.eu1 = e1 - 53;
            n.Pprime = Pprime;
            n.t = t;
            n.gN = double((1.0L + 3.0L * u64) * std::ldexp(1.0L, 1 + clr) * (N + 2) * u64 * u64 *
                          (long double)rho * PL) * (1.0 + 0x1p-40);
            const int eg = clr + (r.bits() - 1) - 52;
            n.g = std::ldexp(1.0, eg);
            n.sh = eg - n.eu1;
            {   // Q = rint(P_inv C'(1)) from C'(1) = H g, |H| < 2^53: the estimate
                // (H >> 22) kq 2^-sq of H g / P (kq < 2^31, the product below 2^61)
                // is within err of it; FP64's P_inv C'(1) is within ymax 2^-51.  The
                // kernel takes the estimate's nearest integer unless it lies within
                // 2^-14 of a half-integer, so err + ymax 2^-51 <= 2^-15 is required.
                const long double ymax = std::ldexp(1.0L, 53 + eg) / PL;
                int sq = 61;
                long double K = 0;
                for (; sq >= 16; sq--) {
                    K = std::rint(std::ldexp(1.0L, 22 + eg + sq) / PL);
                    if (K < 0x1p31L - 1 && ymax * std::ldexp(1.0L, sq) < 0x1p61L) break;
                }
                n.kq = int(K);
                n.sq = sq;
                const long double err = std::ldexp(1.0L, 22 + eg) / PL +
                                        ymax * std::fabs(K * PL / std::ldexp(1.0L, 22 + eg + sq) - 1.0L);
                T.sums_fit &= N < 2 || (n.sh >= 0 && n.sh < 64 && sq >= 16 && err + ymax * 0x1p-51L <= 0x1p-15L);
            }
            n.offset = offset;
            for (int l = 0; l < N; l++) {
                const Big &xl = x[size_t(l)];
                uint64_t s1i;
                double s2;
                if (eg >= 0) { s1i = xl.shr(eg).u64(); s2 = to_double(xl.low(eg)); }
                else { s1i = xl.shl(-eg).u64(); s2 = 0.0; }
                T.s1i[offset + l] = (long long)s1i;
                T.s1d[offset + l] = std::ldexp(double(s1i), eg);
                T.s2d[offset + l] = s2;
            }
        }
        {   // b = 32
            NTable &n = T.n32[N];
            n.P1 = P1;
            n.P2 = 0.0;
            n.Pinv = Pinv;
            n.Pprime = Pprime;
            n.t = t;
            n.gN = double((1.0L + u32) * (N + 2) * u64 * (long double)rho * PL) * (1.0 + 0x1p-40);
            n.g = 1.0;
            n.offset = offset;
            for (int l = 0; l < N; l++) T.s1f[offset + l] = to_double(x[size_t(l)]);
        }
        T.n64[N].eg = std::ilogb(T.n64[N].g);
        T.sums_fit &= split_on_grid(T.s2d + offset, N, T.ks64 + offset, &T.n64[N].esum);
        T.sums_fit &= split_on_grid(T.s1f + offset, N, T.ks32 + offset, &T.n32[N].esum);
        for (int l = 0; l < N; l++) {
            const uint64_t v = uint64_t(T.s1i[offset + l]);
            T.sums_fit &= v < (uint64_t(1) << 62);
            T.s1s[offset + l][0] = int(v & 0x7FFFFFFFu);
            T.s1s[offset + l][1] = int(v >> 31);
        }
        {   // the CRT kernel sums s1.y W_l in 32 bits and forms H = sum s_l1 W_l / g
            // in 64: both bounds with |W_l| <= 128
            long long hy = 0;
            long double h = 0;
            for (int l = 0; l < N; l++) {
                hy += 128ll * T.s1s[offset + l][1];
                h += 128.0L * (long double)T.s1i[offset + l];
            }
            T.sums_fit &= hy < (1ll << 31) && h < 0x1p62L && T.n64[N].eg + 62 < 1023 && T.n64[N].eg > -960;
            // |H| < 2^53 (Lemma 2), which the kernel's integer steps rely on:
            // |W_l| <= floor(p_l / 2)
            long double hb = 0;
            for (int l = 0; l < N; l++) hb += (long double)(kModuli[l] / 2) * (long double)T.s1i[offset + l];
            T.sums_fit &= N < 2 || (hb < 0x1p53L && T.n64[N].esum >= -1022);
            // the dp2a form rebuilds H from three 16-bit piece sums modulo 2^64, which is
            // exact while |H| < 2^63; each piece sum stays below 2^16 128 49 < 2^31, and
            // the fourth piece of every s_l1 / g is zero
            T.sums_fit &= h < 0x1p62L;
            for (int l = 0; l < N; l++) T.sums_fit &= uint64_t(T.s1i[offset + l]) < (uint64_t(1) << 48);
        }
        {   // 16-bit pieces of the constants, two planes per word (the last pair of
            // an odd N pairs its plane with a zero)
            if (poff + (N + 1) / 2 > kPairsLen) { T.sums_fit = false; break; }
            T.n64[N].poff = T.n32[N].poff = poff;
            auto whole = [](const int (*k)[2], int l) { return (uint64_t(uint32_t(k[l][1])) << 31) | uint32_t(k[l][0]); };
            for (int i = 0; 2 * i < N; i++) {
                for (int h = 0; h < 2; h++) {
                    const int l = 2 * i + h;
                    const uint64_t c1 = l < N ? uint64_t(T.s1i[offset + l]) : 0;
                    const uint64_t c2 = l < N ? whole(T.ks64 + offset, l) : 0;
                    const uint64_t c3 = l < N ? whole(T.ks32 + offset, l) : 0;
                    for (int j = 0; j < 4; j++) {
                        T.dp64[poff + i][j] |= uint32_t((c1 >> (16 * j)) & 0xFFFFu) << (16 * h);
                        T.dp64[poff + i][4 + j] |= uint32_t((c2 >> (16 * j)) & 0xFFFFu) << (16 * h);
                        T.dp32[poff + i][j] |= uint32_t((c3 >> (16 * j)) & 0xFFFFu) << (16 * h);
                    }
                }
            }
            poff += (N + 1) / 2;
        }
        offset += N;
    }
}

}  // namespace

const Tables &tables() {
    static Tables T;
    static std::once_flag once;
    std::call_once(once, [] { build(T); });
    return T;
}

}  // namespace oz2
