// Shared device/host definitions of the GB300 GIRG / HRG generator.
//
// Philox4x32-10 (Salmon et al., SC'11), the uniform mapping, and the FP64
// arithmetic that decides edges.  Every FP64 value that decides an edge is
// evaluated with IEEE +, -, *, / and sqrt in a fixed order with no FMA
// contraction (device: __d*_rn intrinsics; host: built with
// -ffp-contract=off), and with elementary functions written here from their
// series (ln via 2 atanh((m-1)/(m+1)) after reduction by powers of two, exp
// via reduction by ln 2 and the Taylor series, sin(pi x) via Taylor series),
// so that host and device -- and any other IEEE machine following the same
// steps -- produce identical bits.
#pragma once
#include <mutex>
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <string.h>

#ifdef __CUDACC__
#define GG_HD __host__ __device__ __forceinline__
#else
#define GG_HD inline
#endif

#if defined(__CUDA_ARCH__)
#define DADD(a, b) __dadd_rn((a), (b))
#define DSUB(a, b) __dsub_rn((a), (b))
#define DMUL(a, b) __dmul_rn((a), (b))
#define DDIV(a, b) __ddiv_rn((a), (b))
#define DSQRT(a) __dsqrt_rn((a))
#else
#define DADD(a, b) ((a) + (b))
#define DSUB(a, b) ((a) - (b))
#define DMUL(a, b) ((a) * (b))
#define DDIV(a, b) ((a) / (b))
#define DSQRT(a) sqrt((a))
#endif

namespace gg {

// Philox counter tags (one stream family per purpose).
constexpr uint32_t kTagWeight = 0x57454947u;
constexpr uint32_t kTagPos = 0x504F5349u;
constexpr uint32_t kTagRadius = 0x52414449u;
constexpr uint32_t kTagPair = 0x50414952u;
constexpr uint32_t kTagJump = 0x2A4Du;  // 14 bits at bit 18 of a stream's second counter word

constexpr int kMaxLayers = 64;
constexpr int kMaxDim = 8;
constexpr int kMaxLevel = 32;

// ---------------------------------------------------------------- Philox
struct P4 {
    uint32_t x, y, z, w;
};

GG_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Philox4x32-10: ten rounds of two 32x32->64 multiplications and xors with a
// Weyl-sequence key schedule.
GG_HD P4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = mulhi32(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = mulhi32(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return P4{c0, c1, c2, c3};
}

// U = (2 (bits >> 12) + 1) 2^-53 in (0,1), bits = hi << 32 | lo.
GG_HD double uniform53(uint32_t lo, uint32_t hi) {
    const uint64_t bits = ((uint64_t)hi << 32) | lo;
    return (double)(2 * (bits >> 12) + 1) * 0x1p-53;
}

// ---------------------------------------------------------------- bit helpers
GG_HD double bits_to_double(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double r;
    memcpy(&r, &b, 8);
    return r;
#endif
}
GG_HD uint64_t double_to_bits(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

GG_HD double pow2i(int k) {  // exact 2^k for -1022 <= k <= 1023
    return bits_to_double((uint64_t)(k + 1023) << 52);
}
GG_HD double dnan() { return bits_to_double(0x7ff8000000000000ULL); }
GG_HD double dinf() { return bits_to_double(0x7ff0000000000000ULL); }

// ---------------------------------------------------------------- det math
constexpr double kPi = 0x1.921fb54442d18p+1;

// 2 atanh(s) = 2 (s + s^3/3 + ... + s^25/25) for |s| <= 0.18.
GG_HD double two_atanh(double s) {
    const double z = DMUL(s, s);
    double p = 1.0 / 25.0;
    p = DADD(1.0 / 23.0, DMUL(z, p));
    p = DADD(1.0 / 21.0, DMUL(z, p));
    p = DADD(1.0 / 19.0, DMUL(z, p));
    p = DADD(1.0 / 17.0, DMUL(z, p));
    p = DADD(1.0 / 15.0, DMUL(z, p));
    p = DADD(1.0 / 13.0, DMUL(z, p));
    p = DADD(1.0 / 11.0, DMUL(z, p));
    p = DADD(1.0 / 9.0, DMUL(z, p));
    p = DADD(1.0 / 7.0, DMUL(z, p));
    p = DADD(1.0 / 5.0, DMUL(z, p));
    p = DADD(1.0 / 3.0, DMUL(z, p));
    double t = DMUL(s, z);
    t = DMUL(t, p);
    return DADD(DMUL(2.0, s), DMUL(2.0, t));
}

// ---------------------------------------------------------------- fixed-point log / exp
// det_log and det_exp work in 64- and 128-bit integers: every step is exact integer
// arithmetic with a stated truncation, so any two implementations of the same steps
// agree bit for bit, and the FP64 units (slow on this GPU) are used only for the
// reduction index of exp.  Q-notation: Qn holds v as round-or-floor(v 2^n).
//   ln x: x = m 2^e, m in (sqrt(1/2), sqrt(2)]; j = round(64 m) in [45, 91]; with
//   D = 64 m - j (exact), r = D / j (Q63: exact for j = 64, else |D| 2^63 times
//   ceil(2^64/j), top 64 bits, sign of D); ln(1 + r) = r P(r), P(r) = sum_k (-r)^k/(k+1)
//   to r^8 by Horner in Q62 with coefficients round(2^62/k); ln x = e ln 2 + ln(j/64)
//   + r P in Q116 (r P from the exact Q125 product, floor-shifted), rounded once to double.
//   e^x (|x| <= 700): k = floor(64 x / ln 2 + 1/2) in FP64, x in Q116 (truncated),
//   r = x - k ln2/64 in Q116, then Q62 (floor); e^r to r^7 by Horner in Q62 with
//   round(2^62/i!), times 2^(j/64) (Q62, j = k mod 64), floor-shifted to Q62, rounded
//   once to double and scaled by 2^((k - j)/64).
// Tables (host, at first use): ln 2 and ln(j/64) = 2 atanh((j-64)/(j+64)) by their
// series in Q124 (terms s^(2i+1)/(2i+1) until zero, each product floor-shifted, each
// quotient truncated), rounded to Q116; 2^(j/64) = e^(j (ln2_Q124 >> 6) 2^-124) by the
// series in Q124 (term_i = floor(term_{i-1} y / 2^124) / i until zero), rounded to Q62.
typedef unsigned __int128 u128;
typedef __int128 i128;

struct DetTab {
    uint64_t lnc_lo[47], lnc_hi[47];  // ln(j/64) in Q116, j = 45..91 (two's complement)
    uint64_t rj[47];                  // ceil(2^64 / j)
    uint64_t e2[64];                  // 2^(j/64) in Q62
    uint64_t ln2_lo, ln2_hi;          // ln 2 in Q116
    uint64_t ln2s_lo, ln2s_hi;        // ln 2 / 64 in Q116
};

GG_HD i128 make_i128(uint64_t lo, uint64_t hi) { return (i128)(((u128)hi << 64) | lo); }

// round(2^62 / k) (ties up)
__host__ __device__ constexpr int64_t q62_recip(int64_t k) {
    return ((int64_t)1 << 62) / k + (((((int64_t)1 << 62) % k) * 2 >= k) ? 1 : 0);
}

// c - floor(a t / 2^sh) and c + floor(a t / 2^sh) for the Horner steps
GG_HD int64_t fx_sub(int64_t c, int64_t a, int64_t t, int sh) {
    return c - (int64_t)(((i128)a * t) >> sh);
}
GG_HD int64_t fx_add(int64_t c, int64_t a, int64_t t, int sh) {
    return c + (int64_t)(((i128)a * t) >> sh);
}

// (a b) >> 124 for a, b < 2^126 (host table construction)
inline u128 mul_q124(u128 a, u128 b) {
    const uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64);
    const uint64_t b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
    const u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
    // 256-bit sum: limbs w0..w3 (64 bits each)
    const u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
    const uint64_t w1 = (uint64_t)mid;
    const u128 hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
    // bits 124 .. 251: hi << 4 | w1 >> 60
    return (hi << 4) | (u128)(w1 >> 60);
}

// 2 atanh(num/den) in Q124 for 0 <= num/den <= 1/3
inline u128 two_atanh_q124(uint64_t num, uint64_t den) {
    const u128 unit = (u128)1 << 124;
    const u128 s = (u128)num * (unit / den) + ((u128)num * (unit % den)) / den;  // floor
    const u128 s2 = mul_q124(s, s);
    u128 p = s, sum = 0;
    for (uint64_t k = 1; p != 0; k += 2) {
        sum += p / k;
        p = mul_q124(p, s2);
    }
    return sum << 1;
}

inline DetTab make_det_tab() {
    DetTab t;
    const u128 ln2 = two_atanh_q124(1, 3);  // ln 2 = 2 atanh(1/3)
    const u128 half8 = (u128)1 << 7, half14 = (u128)1 << 13;
    const u128 l116 = (ln2 + half8) >> 8, ls116 = (ln2 + half14) >> 14;
    t.ln2_lo = (uint64_t)l116;
    t.ln2_hi = (uint64_t)(l116 >> 64);
    t.ln2s_lo = (uint64_t)ls116;
    t.ln2s_hi = (uint64_t)(ls116 >> 64);
    for (int j = 45; j <= 91; ++j) {
        const u128 a = two_atanh_q124((uint64_t)(j > 64 ? j - 64 : 64 - j), (uint64_t)(j + 64));
        const u128 m = (a + half8) >> 8;
        const i128 v = j >= 64 ? (i128)m : -(i128)m;
        t.lnc_lo[j - 45] = (uint64_t)(u128)v;
        t.lnc_hi[j - 45] = (uint64_t)((u128)v >> 64);
        t.rj[j - 45] = (uint64_t)((((u128)1 << 64) + (u128)(j - 1)) / (u128)j);
    }
    const u128 one = (u128)1 << 124, step = ln2 >> 6;
    for (int j = 0; j < 64; ++j) {
        const u128 y = step * (u128)j;
        u128 term = one, sum = 0;
        for (uint64_t i = 1; term != 0; ++i) {
            sum += term;
            term = mul_q124(term, y) / i;
        }
        t.e2[j] = (uint64_t)((sum + ((u128)1 << 61)) >> 62);
    }
    return t;
}

inline const DetTab& det_tab_host() {
    static const DetTab t = make_det_tab();
    return t;
}

#ifdef __CUDACC__
// One device copy per translation unit, filled once per device by det_tables_ready()
// before the first launch of a kernel that uses det_log / det_exp.
static __device__ DetTab g_det_tab;

static inline bool det_tables_ready() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        if (cudaMemcpyToSymbol(g_det_tab, &det_tab_host(), sizeof(DetTab)) != cudaSuccess)
            return false;
        done[dev] = true;
    }
    return true;
}
#endif

GG_HD const DetTab& det_tab() {
#ifdef __CUDA_ARCH__
    return g_det_tab;
#else
    return det_tab_host();
#endif
}

GG_HD int clz128(u128 v) {
    const uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
#ifdef __CUDA_ARCH__
    return hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
#else
    return hi ? __builtin_clzll(hi) : 64 + __builtin_clzll(lo);
#endif
}

// Round |v| 2^-q (v != 0) to the nearest double, ties to even, with the sign of v;
// the result must be a normal number.
GG_HD double fixed_to_double(i128 v, int q) {
    const bool neg = v < 0;
    const u128 u = neg ? (u128)(-v) : (u128)v;
    int p = 127 - clz128(u);  // top bit
    uint64_t m;
    const int sh = p - 52;
    if (sh > 0) {
        m = (uint64_t)(u >> sh);
        const u128 rem = u & (((u128)1 << sh) - 1), half = (u128)1 << (sh - 1);
        if (rem > half || (rem == half && (m & 1))) ++m;
        if (m >> 53) {
            m >>= 1;
            ++p;
        }
    } else {
        m = (uint64_t)(u << -sh);
    }
    const uint64_t b = ((uint64_t)(p - q + 1023) << 52) | (m & 0x000fffffffffffffULL);
    return bits_to_double(neg ? b | 0x8000000000000000ULL : b);
}

// ln x (definition above; NaN for x < 0, -inf at 0, subnormals scaled by 2^54).
GG_HD double det_log(double x) {
    if (x != x || x < 0.0) return dnan();
    if (x == 0.0) return -dinf();
    if (x == dinf()) return dinf();
    int e_adj = 0;
    if (x < 0x1p-1022) {
        x = DMUL(x, 0x1p54);
        e_adj = -54;
    }
    const uint64_t b = double_to_bits(x);
    const uint64_t f = b & 0x000fffffffffffffULL, M = f | 0x0010000000000000ULL;
    int e = (int)(b >> 52) - 1023 + e_adj, s, j;
    if (f > 0x6a09e667f3bcdULL) {  // m > sqrt 2: m = M 2^-53
        s = 53;
        e += 1;
        j = 32 + (int)((f + (1ULL << 46)) >> 47);
    } else {  // m = M 2^-52
        s = 52;
        j = 64 + (int)((f + (1ULL << 45)) >> 46);
    }
    const DetTab& T = det_tab();
    const int64_t D = (int64_t)(M << 6) - ((int64_t)j << s);  // (64 m - j) 2^s
    int64_t r;                                                // Q63
    if (j == 64) {
        r = D * ((int64_t)1 << (57 - s));
    } else {
        const uint64_t N = (uint64_t)(D < 0 ? -D : D) << (63 - s);
        const uint64_t q = (uint64_t)(((u128)N * T.rj[j - 45]) >> 64);
        r = D < 0 ? -(int64_t)q : (int64_t)q;
    }
    // P(r) = 1 - r (1/2 - r (1/3 - ... - r (1/8 - r/9))) in Q62
    int64_t t = q62_recip(9);
    t = fx_sub(q62_recip(8), r, t, 63);
    t = fx_sub(q62_recip(7), r, t, 63);
    t = fx_sub(q62_recip(6), r, t, 63);
    t = fx_sub(q62_recip(5), r, t, 63);
    t = fx_sub(q62_recip(4), r, t, 63);
    t = fx_sub(q62_recip(3), r, t, 63);
    t = fx_sub(q62_recip(2), r, t, 63);
    t = fx_sub(q62_recip(1), r, t, 63);
    const i128 l1 = ((i128)r * t) >> 9;  // r P in Q116 (floor)
    const i128 L = (i128)e * make_i128(T.ln2_lo, T.ln2_hi) +
                   make_i128(T.lnc_lo[j - 45], T.lnc_hi[j - 45]) + l1;
    if (L == 0) return 0.0;
    return fixed_to_double(L, 116);
}

// e^x (definition above; inf above 710, 0 below -746, NaN passes through).
GG_HD double det_exp(double x) {
    if (x != x) return x;
    if (x > 710.0) return dinf();
    if (x < -746.0) return 0.0;
    const double kd = floor(DADD(DMUL(x, 0x1.71547652b82fep+6), 0.5));
    const int k = (int)kd;
    const DetTab& T = det_tab();
    // x in Q116, truncated toward zero
    const uint64_t b = double_to_bits(x);
    const int be = (int)((b >> 52) & 0x7ff);
    i128 X = 0;
    if (be != 0) {
        const uint64_t M = (b & 0x000fffffffffffffULL) | 0x0010000000000000ULL;
        const int sh = be - 1075 + 116;  // x = M 2^(be - 1075)
        u128 u;
        if (sh >= 0)
            u = (u128)M << sh;
        else
            u = sh > -64 ? (u128)(M >> -sh) : (u128)0;
        X = (b >> 63) ? -(i128)u : (i128)u;
    }
    const i128 R = X - (i128)k * make_i128(T.ln2s_lo, T.ln2s_hi);
    const int64_t r = (int64_t)(R >> 54);  // Q62
    // e^r = 1 + r (1 + r (1/2 + r (1/6 + ... + r/5040))) in Q62
    int64_t sacc = q62_recip(5040);
    sacc = fx_add(q62_recip(720), r, sacc, 62);
    sacc = fx_add(q62_recip(120), r, sacc, 62);
    sacc = fx_add(q62_recip(24), r, sacc, 62);
    sacc = fx_add(q62_recip(6), r, sacc, 62);
    sacc = fx_add(q62_recip(2), r, sacc, 62);
    sacc = fx_add(q62_recip(1), r, sacc, 62);
    sacc = fx_add(q62_recip(1), r, sacc, 62);
    const int j = k & 63;
    const int m = (k - j) / 64;
    const uint64_t V = (uint64_t)(((u128)(uint64_t)sacc * T.e2[j]) >> 62);  // Q62
    const double v = fixed_to_double((i128)V, 62);
    if (m > 1023) return DMUL(DMUL(v, pow2i(1023)), pow2i(m - 1023));
    if (m < -1021) return DMUL(DMUL(v, pow2i(m + 600)), pow2i(-600));
    return DMUL(v, pow2i(m));
}

// ln(1+x), x > -1: 2 atanh(x/(2+x)) for |x| <= 1/4, else ln(1+x).
GG_HD double det_log1p(double x) {
    if (x != x || x < -1.0) return dnan();
    if (x == -1.0) return -dinf();
    if (x < -0.25 || x > 0.25) return det_log(DADD(1.0, x));
    return two_atanh(DDIV(x, DADD(2.0, x)));
}


GG_HD double det_pow(double x, double y) { return det_exp(DMUL(y, det_log(x))); }

// sin(pi x), x in [0, 1/2].
GG_HD double det_sinpi(double x) {
    if (x <= 0.25) {
        const double y = DMUL(x, kPi);
        const double z = DMUL(y, y);
        double p = -1.0 / 1307674368000.0;
        p = DADD(1.0 / 6227020800.0, DMUL(z, p));
        p = DADD(-1.0 / 39916800.0, DMUL(z, p));
        p = DADD(1.0 / 362880.0, DMUL(z, p));
        p = DADD(-1.0 / 5040.0, DMUL(z, p));
        p = DADD(1.0 / 120.0, DMUL(z, p));
        p = DADD(-1.0 / 6.0, DMUL(z, p));
        const double t = DMUL(y, z);
        return DADD(y, DMUL(t, p));
    }
    const double y = DMUL(DSUB(0.5, x), kPi);
    const double z = DMUL(y, y);
    double p = 1.0 / 20922789888000.0;
    p = DADD(-1.0 / 87178291200.0, DMUL(z, p));
    p = DADD(1.0 / 479001600.0, DMUL(z, p));
    p = DADD(-1.0 / 3628800.0, DMUL(z, p));
    p = DADD(1.0 / 40320.0, DMUL(z, p));
    p = DADD(-1.0 / 720.0, DMUL(z, p));
    p = DADD(1.0 / 24.0, DMUL(z, p));
    p = DADD(-0.5, DMUL(z, p));
    return DADD(1.0, DMUL(z, p));
}

// acosh z = ln(z + sqrt(z^2 - 1)).
GG_HD double det_acosh(double z) { return det_log(DADD(z, DSQRT(DSUB(DMUL(z, z), 1.0)))); }

// x^(1/d) (d = 1: x).
GG_HD double root_d(double x, int d) {
    if (d == 1) return x;
    return det_exp(DDIV(det_log(x), (double)d));
}

// ---------------------------------------------------------------- the model

// Circular difference of two 32-bit fixed-point coordinates (torus).
GG_HD uint32_t circ_diff(uint32_t a, uint32_t b) {
    const uint32_t t = a - b, u = b - a;
    return t < u ? t : u;
}

// Eq. 1 with the model's scale K = c^T (K = c^d at T = 0), which stays a moderate
// number for every T while c = K^(1/T) leaves the range of doubles as T -> 0:
// x = K q / r^d with q = w_u w_v / W; p = 1 if x >= 1, else x^(1/T) (repeated
// products when 1/T is an integer).
GG_HD double girg_p_at(double wu, double wv, double r, double W, double K, double invT, int m_int,
                       int d) {
    const double q = DDIV(DMUL(wu, wv), W);
    double rd = r;
    for (int k = 1; k < d; ++k) rd = DMUL(rd, r);
    const double x = DDIV(DMUL(K, q), rd);
    if (x >= 1.0) return 1.0;
    double p;
    if (m_int > 0) {
        p = x;
        for (int k = 1; k < m_int; ++k) p = DMUL(p, x);
    } else {
        p = det_exp(DMUL(invT, det_log(x)));
    }
    return p;
}

// Eq. 1 at the fixed-point distance D (r = D 2^-32; r = 0 gives p = 1).
GG_HD double girg_p64(double wu, double wv, uint32_t D, double W, double K, double invT, int m_int,
                      int d) {
    if (D == 0) return 1.0;
    return girg_p_at(wu, wv, (double)D * 0x1p-32, W, K, invT, m_int, d);
}

// Threshold variant: edge iff r^d <= K w_u w_v / W (r <= c (w_u w_v / W)^(1/d)).
GG_HD bool girg_thresh64(double wu, double wv, uint32_t D, double W, double K, int d) {
    const double q = DDIV(DMUL(wu, wv), W);
    const double r = (double)D * 0x1p-32;
    double rd = r;
    for (int k = 1; k < d; ++k) rd = DMUL(rd, r);
    return rd <= DMUL(K, q);
}

// The scale K of the c of Eq. 1: c^T (T > 0) or c^d (T = 0).
GG_HD double girg_K_of_c(double c, int d, double T) {
    if (T > 0.0) return det_pow(c, T);
    double k = c;
    for (int i = 1; i < d; ++i) k = DMUL(k, c);
    return k;
}

// cosh of the hyperbolic distance: cosh(r_u - r_v) + 2 sinh r_u sinh r_v sin^2(pi D 2^-32)
// from E = e^r and sh = sinh r of both vertices.
GG_HD double hrg_coshd64(double Eu, double shu, double Ev, double shv, uint32_t D) {
    const double s = det_sinpi((double)D * 0x1p-32);
    const double ch = DMUL(DADD(DDIV(Eu, Ev), DDIV(Ev, Eu)), 0.5);
    double t = DMUL(shu, shv);
    t = DMUL(t, DMUL(s, s));
    return DADD(ch, DMUL(2.0, t));
}

GG_HD void hrg_vertex64(double r, double* E, double* sh) {
    *E = det_exp(r);
    *sh = DMUL(DSUB(*E, DDIV(1.0, *E)), 0.5);
}

// p_T(d) = 1 / (exp((d - R) / 2T) + 1) from cosh d.
GG_HD double hrg_p_from_coshd(double coshd, double R, double T) {
    const double dist = det_acosh(coshd);
    return DDIV(1.0, DADD(det_exp(DDIV(DSUB(dist, R), DMUL(2.0, T))), 1.0));
}

// Bucket of a weight: floor(log2(w / w_min)) from the exponent of the quotient.
GG_HD int layer_of(double w, double w_min) {
    const double ratio = DDIV(w, w_min);
    const int eb = (int)((double_to_bits(ratio) >> 52) & 0x7ff);
    int layer = eb - 1023;
    if (layer < 0) layer = 0;
    if (layer > kMaxLayers - 1) layer = kMaxLayers - 1;
    return layer;
}

// Chunk length exponent k of a geometric-jump stream under bound pbar:
// 2^k pbar in [4, 8), k clamped to [3, 31].
GG_HD int chunk_log(double pbar) {
    const int eb = (int)((double_to_bits(pbar) >> 52) & 0x7ff);
    const int e = eb - 1022;  // pbar = m 2^e, m in [0.5, 1) (pbar is normal here)
    int k = 3 - e;
    if (k < 3) k = 3;
    if (k > 31) k = 31;
    return k;
}

}  // namespace gg
