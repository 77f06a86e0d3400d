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
constexpr double kLn2Hi = 0x1.62e42fee00000p-1;   // ln 2 rounded to 32 bits
constexpr double kLn2Lo = 0x1.a39ef35793c76p-33;  // ln 2 - kLn2Hi
constexpr double kInvLn2 = 0x1.71547652b82fep+0;
constexpr double kPi = 0x1.921fb54442d18p+1;
constexpr double kSqrt2 = 0x1.6a09e667f3bcdp+0;

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

// ln x by the series: x = m 2^e with m in (sqrt(1/2), sqrt(2)], ln m = 2 atanh((m-1)/(m+1)).
// Only builds the tables of det_log / det_exp below.
GG_HD double det_log_series(double x) {
    if (x != x || x < 0.0) return dnan();
    if (x == 0.0) return -dinf();
    if (x == dinf()) return dinf();
    int e_adj = 0;
    if (x < 0x1p-1022) {
        x = DMUL(x, 0x1p54);
        e_adj = -54;
    }
    uint64_t b = double_to_bits(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = bits_to_double((b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL);
    if (m > kSqrt2) {
        m = DMUL(m, 0.5);
        e = e + 1;
    }
    e = e + e_adj;
    const double s = DDIV(DSUB(m, 1.0), DADD(m, 1.0));
    const double lm = two_atanh(s);
    const double ed = (double)e;
    return DADD(DMUL(ed, kLn2Hi), DADD(lm, DMUL(ed, kLn2Lo)));
}

// e^x = 2^k e^r, k = round(x / ln 2), r = x - k ln 2, Taylor series to r^17.
GG_HD double det_exp_series(double x) {
    if (x != x) return x;
    if (x > 710.0) return dinf();
    if (x < -746.0) return 0.0;
    const double kd = floor(DADD(DMUL(x, kInvLn2), 0.5));
    const int k = (int)kd;
    const double r = DSUB(DSUB(x, DMUL(kd, kLn2Hi)), DMUL(kd, kLn2Lo));
    double p = 1.0 / 355687428096000.0;
    p = DADD(1.0 / 20922789888000.0, DMUL(r, p));
    p = DADD(1.0 / 1307674368000.0, DMUL(r, p));
    p = DADD(1.0 / 87178291200.0, DMUL(r, p));
    p = DADD(1.0 / 6227020800.0, DMUL(r, p));
    p = DADD(1.0 / 479001600.0, DMUL(r, p));
    p = DADD(1.0 / 39916800.0, DMUL(r, p));
    p = DADD(1.0 / 3628800.0, DMUL(r, p));
    p = DADD(1.0 / 362880.0, DMUL(r, p));
    p = DADD(1.0 / 40320.0, DMUL(r, p));
    p = DADD(1.0 / 5040.0, DMUL(r, p));
    p = DADD(1.0 / 720.0, DMUL(r, p));
    p = DADD(1.0 / 120.0, DMUL(r, p));
    p = DADD(1.0 / 24.0, DMUL(r, p));
    p = DADD(1.0 / 6.0, DMUL(r, p));
    p = DADD(0.5, DMUL(r, p));
    p = DADD(1.0, DMUL(r, p));
    p = DADD(1.0, DMUL(r, p));
    if (k > 1023) return DMUL(DMUL(p, pow2i(1023)), pow2i(k - 1023));
    if (k < -1021) return DMUL(DMUL(p, pow2i(k + 600)), pow2i(-600));
    return DMUL(p, pow2i(k));
}

// ---------------------------------------------------------------- table-driven log / exp
// Tables of the deterministic log and exp, built from the series forms above (the
// same IEEE operations on every machine, so every copy holds the same bits):
// e2[j] = 2^(j/64), j = 0..63; lc[j - 45] = ln(j/64), ic[j - 45] = 64/j, j = 45..91.
struct DetTab {
    double e2[64];
    double lc[47];
    double ic[47];
};

inline DetTab make_det_tab() {
    DetTab t;
    for (int j = 0; j < 64; ++j)
        t.e2[j] = det_exp_series(DADD(DMUL((double)j, 0x1.62e42fee00000p-7),
                                      DMUL((double)j, 0x1.a39ef35793c76p-39)));
    for (int j = 45; j <= 91; ++j) {
        t.lc[j - 45] = det_log_series((double)j * 0x1p-6);
        t.ic[j - 45] = 64.0 / (double)j;
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

// ln x: x = m 2^e with m in (sqrt(1/2), sqrt(2)]; m = c (1 + r) with c = j/64 the
// nearest table point, r = (m - c) 64/j (m - c is exact), |r| <= 1/90; ln(1 + r) by
// its series to r^9.  ln x = e ln 2 + ln c + ln(1 + r).
GG_HD double det_log(double x) {
#ifdef __CUDA_ARCH__
    {
        // positive normal x: the same operations, with the classification, the choice
        // of m and the index j taken from the bits (integer units, not the FP64 pipe);
        // j = floor(64 m + 1/2) is (f + 2^45) >> 46 above 1 and (f + 2^46) >> 47 below,
        // f the fraction bits, since 64 m + 1/2 is exact or rounds within its integer
        const uint64_t b = double_to_bits(x);
        if (b - 0x0010000000000000ULL < 0x7FE0000000000000ULL) {
            const uint64_t f = b & 0x000fffffffffffffULL;
            int e = (int)(b >> 52) - 1023, j;
            double m, c;
            if (f > 0x6a09e667f3bcdULL) {  // m > sqrt 2: m / 2 in (sqrt 1/2, 1)
                m = bits_to_double(f | 0x3fe0000000000000ULL);
                e = e + 1;
                j = 32 + (int)((f + (1ULL << 46)) >> 47);
            } else {
                m = bits_to_double(f | 0x3ff0000000000000ULL);
                j = 64 + (int)((f + (1ULL << 45)) >> 46);
            }
            c = j < 64 ? bits_to_double(0x3fe0000000000000ULL | ((uint64_t)(j - 32) << 47))
                       : bits_to_double(0x3ff0000000000000ULL | ((uint64_t)(j - 64) << 46));
            const DetTab& T = det_tab();
            const double r = DMUL(DSUB(m, c), T.ic[j - 45]);
            double t = 1.0 / 9.0;
            t = DSUB(1.0 / 8.0, DMUL(r, t));
            t = DSUB(1.0 / 7.0, DMUL(r, t));
            t = DSUB(1.0 / 6.0, DMUL(r, t));
            t = DSUB(1.0 / 5.0, DMUL(r, t));
            t = DSUB(1.0 / 4.0, DMUL(r, t));
            t = DSUB(1.0 / 3.0, DMUL(r, t));
            t = DSUB(0.5, DMUL(r, t));
            t = DSUB(1.0, DMUL(r, t));
            const double l1 = DMUL(r, t);
            const double ed = (double)e;
            return DADD(DMUL(ed, kLn2Hi), DADD(T.lc[j - 45], DADD(l1, DMUL(ed, kLn2Lo))));
        }
    }
#endif
    if (x != x || x < 0.0) return dnan();
    if (x == 0.0) return -dinf();
    if (x == dinf()) return dinf();
    int e_adj = 0;
    if (x < 0x1p-1022) {
        x = DMUL(x, 0x1p54);
        e_adj = -54;
    }
    const uint64_t b = double_to_bits(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = bits_to_double((b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL);
    if (m > kSqrt2) {
        m = DMUL(m, 0.5);
        e = e + 1;
    }
    e = e + e_adj;
    const int j = (int)floor(DADD(DMUL(m, 64.0), 0.5));
    const DetTab& T = det_tab();
    const double r = DMUL(DSUB(m, (double)j * 0x1p-6), T.ic[j - 45]);
    double t = 1.0 / 9.0;
    t = DSUB(1.0 / 8.0, DMUL(r, t));
    t = DSUB(1.0 / 7.0, DMUL(r, t));
    t = DSUB(1.0 / 6.0, DMUL(r, t));
    t = DSUB(1.0 / 5.0, DMUL(r, t));
    t = DSUB(1.0 / 4.0, DMUL(r, t));
    t = DSUB(1.0 / 3.0, DMUL(r, t));
    t = DSUB(0.5, DMUL(r, t));
    t = DSUB(1.0, DMUL(r, t));
    const double l1 = DMUL(r, t);
    const double ed = (double)e;
    return DADD(DMUL(ed, kLn2Hi), DADD(T.lc[j - 45], DADD(l1, DMUL(ed, kLn2Lo))));
}

// e^x = 2^m 2^(j/64) e^r with k = round(64 x / ln 2) = 64 m + j, r = x - k ln2/64
// (|r| <= ln2/128), e^r by its series to r^7.
GG_HD double det_exp(double x) {
#ifdef __CUDA_ARCH__
    // |x| <= 700 (the integer test covers NaN): the same operations without the range
    // checks; there m = floor(k / 64) lies in [-1011, 1010], a normal power of two
    if ((double_to_bits(x) & 0x7fffffffffffffffULL) <= 0x4085e00000000000ULL) {
        const double kd = floor(DADD(DMUL(x, 0x1.71547652b82fep+6), 0.5));
        const int k = (int)kd;
        const double r =
            DSUB(DSUB(x, DMUL(kd, 0x1.62e42fee00000p-7)), DMUL(kd, 0x1.a39ef35793c76p-39));
        const int j = k & 63;
        const int m = (k - j) / 64;
        double p = 1.0 / 5040.0;
        p = DADD(1.0 / 720.0, DMUL(r, p));
        p = DADD(1.0 / 120.0, DMUL(r, p));
        p = DADD(1.0 / 24.0, DMUL(r, p));
        p = DADD(1.0 / 6.0, DMUL(r, p));
        p = DADD(0.5, DMUL(r, p));
        p = DADD(1.0, DMUL(r, p));
        p = DADD(1.0, DMUL(r, p));
        return DMUL(DMUL(det_tab().e2[j], p), pow2i(m));
    }
#endif
    if (x != x) return x;
    if (x > 710.0) return dinf();
    if (x < -746.0) return 0.0;
    const double kd = floor(DADD(DMUL(x, 0x1.71547652b82fep+6), 0.5));
    const int k = (int)kd;
    const double r = DSUB(DSUB(x, DMUL(kd, 0x1.62e42fee00000p-7)), DMUL(kd, 0x1.a39ef35793c76p-39));
    const int j = k & 63;
    const int m = (k - j) / 64;
    double p = 1.0 / 5040.0;
    p = DADD(1.0 / 720.0, DMUL(r, p));
    p = DADD(1.0 / 120.0, DMUL(r, p));
    p = DADD(1.0 / 24.0, DMUL(r, p));
    p = DADD(1.0 / 6.0, DMUL(r, p));
    p = DADD(0.5, DMUL(r, p));
    p = DADD(1.0, DMUL(r, p));
    p = DADD(1.0, DMUL(r, p));
    const double v = DMUL(det_tab().e2[j], p);
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
