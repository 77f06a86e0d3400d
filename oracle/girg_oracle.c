/*
 * CPU oracle for the GIRG / HRG sampler of Blaesius, Friedrich, Katzmann,
 * Meyer, Penschuck and Weyand, "Efficiently Generating Geometric
 * Inhomogeneous and Hyperbolic Random Graphs" (arXiv 1905.06706).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
 * leg of the benchmark call this file to check the CUDA library; the
 * library never calls it, and the two share no code, header or constant
 * table.  Everything here is plain, sequential FP64 C, written for a reader
 * to check against the paper by eye, not for speed.
 *
 * Contents
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
 *     generator both sides implement from its published definition.
 *   - det_log / det_exp: ln and exp in 64/128-bit fixed point (argument
 *     reduction by powers of two and a 64-entry table, then the series of
 *     ln(1 + r) and e^r), every truncation specified and the result rounded
 *     once, so any implementation of the same integer steps reproduces them bit
 *     for bit; det_log1p / det_sinpi / det_acosh / det_pow build on them with
 *     IEEE +, -, *, / in a fixed order (FMA contraction disabled).  The CUDA
 *     library implements the same fixed-point method on its own, so that the
 *     default build of this file and the library take identical decisions and
 *     their edge sets are compared for equality.
 *   - The plain build (compiled with -DORC_PLAIN): the same file with the C
 *     library's log, exp, log1p, pow, sin and acosh in place of the det_*
 *     functions, and nothing else changed.  It shares no arithmetic with the
 *     CUDA library beyond IEEE +, -, *, /; the library's edge sets are checked
 *     against it at a tolerance on flipped decisions, using the decision audit
 *     (every decision within a relative eps of its threshold is recorded).
 *   - Model inputs: Pareto weights (Sec. 2.1, Sec. 5.1 step 1), uniform torus
 *     positions in 32-bit fixed point (Sec. 2.1), HRG radii and angles
 *     (Sec. 2.2) and the HRG->GIRG mapping (Sec. 2.3).
 *   - Eq. 1 and its threshold variant (Sec. 2.1); the HRG connection
 *     probability p_T(d) (Sec. 2.2) with cosh d in the cancellation-free form
 *     cosh(r_u - r_v) + 2 sinh r_u sinh r_v sin^2(dtheta/2).
 *   - Oracle 1: the quadratic all-pairs generator (Table 1, "Pairwise").
 *   - Oracle 2: the cell-pair sampler, Algorithm 1 (Sec. 3.3) run
 *     recursively from the root pair, with weight buckets and levels
 *     (Sec. 3.1), geometric jumps (Sec. 3.2), Morton order and prefix sums
 *     (Sec. 3.4, Lemma 1) and the double-counting rules (App. B.1).
 *   - The expected-average-degree formula and the binary search for c
 *     (Sec. 4.1, App. B.2).
 *
 * Parity unpinned: none of the functions here lacks a pin in
 * tests/test_oracle_*.py (Philox by the Random123 known-answer vectors and an
 * independent implementation, the elementary functions against libm and
 * mpmath, the samplers by brute-force partition, bound and binomial tests,
 * the degree formula by numerical integration and Monte Carlo).
 *
 * Conventions shared with the CUDA library (each side implements them on
 * its own):
 *   key of every Philox call  = (seed_lo, seed_hi) unless stated otherwise
 *   uniform from two words    = (2*(bits64 >> 12) + 1) * 2^-53  in (0,1),
 *                               bits64 = hi << 32 | lo
 *   weight of vertex v        = w_min * U^(-1/(beta-1)),
 *                               U from ctr (v_lo, v_hi, TAG_WEIGHT, 0)
 *   coordinate k of vertex v  = word (k mod 4) of ctr (v_lo, v_hi, TAG_POS, k/4)
 *   HRG radius of vertex v    = acosh(1 + U (cosh(alpha R) - 1)) / alpha,
 *                               U from ctr (v_lo, v_hi, TAG_RADIUS, 0)
 *   type-I coin of pair u<v   = U from words 0,1 of ctr (u, v, TAG_PAIR, 0)
 *   type-II streams           = for a cell A of bucket i at level l, bucket j and gap g,
 *                               one geometric-jump stream over V_i^A x (the concatenation
 *                               of V_j^B over its distant partner cells B with gap g, in
 *                               increasing rank of B, see t2_rank); chunks of 2^k
 *                               indices, 2^k pbar in [4, 8), k in [3, 31]
 *   type-II draw t of chunk h = ctr (A, l|i<<5|j<<11|(g-1)<<17|TAG_JUMP<<18, h, t):
 *                               words 0,1 -> jump uniform, words 2,3 -> acceptance
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define TAG_WEIGHT 0x57454947u
#define TAG_POS 0x504F5349u
#define TAG_RADIUS 0x52414449u
#define TAG_PAIR 0x50414952u
#define TAG_JUMP 0x2A4Du /* 14 bits; sets bit 31 of the second counter word */

#define MAXL 64 /* weight layers */
#define MAXD 8  /* dimensions */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4 and the Random123 reference)  */
/* ------------------------------------------------------------------------ */

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* Weyl increments of the key schedule */
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static void philox_seed(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                        uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* Uniform in (0,1) on the grid of odd multiples of 2^-53. */
double orc_uniform(uint32_t lo, uint32_t hi) {
    uint64_t bits = ((uint64_t)hi << 32) | lo;
    return (double)(2 * (bits >> 12) + 1) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* Deterministic elementary functions                                         */
/* ------------------------------------------------------------------------ */

#ifdef ORC_PLAIN
/* The plain build (-DORC_PLAIN): the elementary functions are the C library's own
 * log, exp, log1p, pow, sin and acosh, with no table or series of this file, so the
 * samplers below evaluate Eq. 1, p_T(d) and the geometric jumps of Sec. 3.2 exactly as
 * the paper writes them, up to the library's rounding.  The CUDA library's edge sets
 * are checked against this build at a stated tolerance on the flipped decisions (each
 * flip within a relative 1e-12 of its threshold, see the decision audit below). */
double orc_det_log(double x) { return log(x); }
double orc_det_exp(double x) { return exp(x); }
double orc_det_log1p(double x) { return log1p(x); }
double orc_det_pow(double x, double y) { return pow(x, y); }
double orc_det_sinpi(double x) { return sin(M_PI * x); }
double orc_det_acosh(double z) { return acosh(z); }
#else
static const double PI_D = 0x1.921fb54442d18p+1;

static double pow2i(int k) { /* exact 2^k for -1022 <= k <= 1023 */
    uint64_t bits = (uint64_t)(k + 1023) << 52;
    double r;
    memcpy(&r, &bits, 8);
    return r;
}

/* 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), |s| <= 0.18, 12 terms. */
static double two_atanh_series(double s) {
    double z = s * s;
    double p = 1.0 / 25.0;
    p = 1.0 / 23.0 + z * p;
    p = 1.0 / 21.0 + z * p;
    p = 1.0 / 19.0 + z * p;
    p = 1.0 / 17.0 + z * p;
    p = 1.0 / 15.0 + z * p;
    p = 1.0 / 13.0 + z * p;
    p = 1.0 / 11.0 + z * p;
    p = 1.0 / 9.0 + z * p;
    p = 1.0 / 7.0 + z * p;
    p = 1.0 / 5.0 + z * p;
    p = 1.0 / 3.0 + z * p;
    double t = s * z;
    t = t * p;
    return 2.0 * s + 2.0 * t;
}

/* Fixed-point ln and exp.  Every step is integer arithmetic with a stated rounding,
 * so an independent implementation of the same steps gives the same bits.
 * Qn: the integer v 2^n.  u128 / i128: unsigned / signed 128-bit integers.
 *
 * ln x, x = m 2^e with m in (sqrt(1/2), sqrt(2)] (the significand halved when it
 * exceeds sqrt 2): j = round(64 m) in [45, 91]; D = (64 m - j) 2^s exactly (s = 52 or
 * 53, the significand's scale); r = D / (j 2^s) in Q63, exactly D 2^(57-s) when j = 64,
 * else the top 64 bits of |D| 2^(63-s) ceil(2^64/j) with the sign of D; P(r) =
 * 1 - r/2 + r^2/3 - ... + r^8/9 by Horner in Q62 (coefficients round(2^62/k), each
 * product floor-shifted by 63); ln x = e ln2 + ln(j/64) + floor(r P 2^-9) in Q116,
 * rounded once to the nearest double (ties to even).
 *
 * e^x, |x| <= 710: k = floor(64 x / ln 2 + 1/2) in double arithmetic; x in Q116
 * (truncated toward zero); r = x - k ln2/64 in Q116, floor-shifted to Q62; e^r =
 * 1 + r + ... + r^7/7! by Horner in Q62 (coefficients round(2^62/i!), products
 * floor-shifted by 62); times 2^(j/64) (Q62, j = k mod 64), floor-shifted to Q62;
 * rounded to the nearest double and scaled by 2^((k - j)/64).
 *
 * Constants: ln 2 = 2 atanh(1/3) and ln(j/64) = +-2 atanh(|j-64|/(j+64)) by the series
 * sum_i s^(2i+1)/(2i+1) in Q124 (s truncated, s^2 and each power floor-shifted, each
 * quotient truncated, until the power is zero), rounded to Q116; 2^(j/64) by the
 * series of e^y, y = j floor(ln2_Q124 / 64), in Q124 (term_i = floor(floor(term_{i-1}
 * y / 2^124) / i) until zero), rounded to Q62. */
typedef unsigned __int128 u128;
typedef __int128 i128;

static i128 FX_LN2, FX_LN2_64;    /* Q116 */
static i128 FX_LNJ[47];            /* ln(j/64), Q116, j = 45..91 */
static uint64_t FX_RJ[47];         /* ceil(2^64 / j) */
static uint64_t FX_E2[64];         /* 2^(j/64), Q62 */
static int64_t FX_LOGC[10];        /* round(2^62 / k), k = 1..9 */
static int64_t FX_EXPC[8];         /* round(2^62 / i!), i = 0..7 */
static int fx_ready = 0;

/* floor(a b / 2^124) for a, b < 2^126: the 256-bit product from four 64x64 parts */
static u128 fx_mul124(u128 a, u128 b) {
    uint64_t al = (uint64_t)a, ah = (uint64_t)(a >> 64);
    uint64_t bl = (uint64_t)b, bh = (uint64_t)(b >> 64);
    u128 ll = (u128)al * bl, lh = (u128)al * bh, hl = (u128)ah * bl, hh = (u128)ah * bh;
    u128 cross = (ll >> 64) + (u128)(uint64_t)lh + (u128)(uint64_t)hl; /* bits 64.. */
    u128 top = hh + (lh >> 64) + (hl >> 64) + (cross >> 64);            /* bits 128.. */
    return (top << 4) + ((uint64_t)cross >> 60);
}

static u128 fx_two_atanh(uint64_t num, uint64_t den) { /* Q124, num/den <= 1/3 */
    u128 one = (u128)1 << 124;
    u128 s = (u128)num * (one / den) + ((u128)num * (one % den)) / den;
    u128 s2 = fx_mul124(s, s);
    u128 acc = 0, pw = s;
    uint64_t k = 1;
    while (pw != 0) {
        acc += pw / k;
        pw = fx_mul124(pw, s2);
        k += 2;
    }
    return 2 * acc;
}

static void fx_init(void) {
    if (fx_ready) return;
    u128 ln2 = fx_two_atanh(1, 3);
    FX_LN2 = (i128)((ln2 + ((u128)1 << 7)) >> 8);
    FX_LN2_64 = (i128)((ln2 + ((u128)1 << 13)) >> 14);
    for (int j = 45; j <= 91; j++) {
        u128 a = fx_two_atanh((uint64_t)(j >= 64 ? j - 64 : 64 - j), (uint64_t)(j + 64));
        i128 v = (i128)((a + ((u128)1 << 7)) >> 8);
        FX_LNJ[j - 45] = j >= 64 ? v : -v;
        FX_RJ[j - 45] = (uint64_t)((((u128)1 << 64) + (u128)(j - 1)) / (u128)j);
    }
    u128 step = ln2 >> 6;
    for (int j = 0; j < 64; j++) {
        u128 y = step * (u128)j, term = (u128)1 << 124, acc = 0;
        for (uint64_t i = 1; term != 0; i++) {
            acc += term;
            term = fx_mul124(term, y) / i;
        }
        FX_E2[j] = (uint64_t)((acc + ((u128)1 << 61)) >> 62);
    }
    int64_t one = (int64_t)1 << 62;
    for (int k = 1; k <= 9; k++) {
        int64_t q = one / k, rem = one % k;
        FX_LOGC[k] = q + (2 * rem >= k ? 1 : 0);
    }
    int64_t f = 1;
    for (int i = 0; i <= 7; i++) {
        if (i > 0) f *= i;
        int64_t q = one / f, rem = one % f;
        FX_EXPC[i] = q + (2 * rem >= f ? 1 : 0);
    }
    fx_ready = 1;
}

static int fx_clz128(u128 v) {
    uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
    return hi ? __builtin_clzll(hi) : 64 + __builtin_clzll(lo);
}

/* nearest double (ties to even) to v 2^-q, v != 0, the result normal */
static double fx_to_double(i128 v, int q) {
    int neg = v < 0;
    u128 u = neg ? (u128)(-v) : (u128)v;
    int top = 127 - fx_clz128(u);
    uint64_t mant;
    int sh = top - 52;
    if (sh > 0) {
        mant = (uint64_t)(u >> sh);
        u128 rest = u - ((u128)mant << sh), half = (u128)1 << (sh - 1);
        if (rest > half || (rest == half && (mant & 1))) mant++;
        if (mant == (1ULL << 53)) {
            mant >>= 1;
            top++;
        }
    } else {
        mant = (uint64_t)(u << (-sh));
    }
    uint64_t bits = ((uint64_t)(top - q + 1023) << 52) | (mant & 0x000fffffffffffffULL);
    if (neg) bits |= 0x8000000000000000ULL;
    double r;
    memcpy(&r, &bits, 8);
    return r;
}

double orc_det_log(double x) {
    if (x != x || x < 0.0) return NAN;
    if (x == 0.0) return -INFINITY;
    if (x == INFINITY) return INFINITY;
    fx_init();
    int e_adj = 0;
    if (x < 0x1p-1022) { /* subnormal: scale into the normal range */
        x = x * 0x1p54;
        e_adj = -54;
    }
    uint64_t bits;
    memcpy(&bits, &x, 8);
    uint64_t frac = bits & 0x000fffffffffffffULL;
    uint64_t sig = frac | 0x0010000000000000ULL; /* m = sig 2^-52 in [1, 2) */
    int e = (int)(bits >> 52) - 1023 + e_adj;
    int s, j;
    if (frac > 0x6a09e667f3bcdULL) { /* m > sqrt 2: use m/2 = sig 2^-53 */
        s = 53;
        e = e + 1;
        j = 32 + (int)((frac + (1ULL << 46)) >> 47);
    } else {
        s = 52;
        j = 64 + (int)((frac + (1ULL << 45)) >> 46);
    }
    int64_t D = (int64_t)(sig * 64) - (int64_t)j * ((int64_t)1 << s);
    int64_t r;
    if (j == 64) {
        r = D * ((int64_t)1 << (57 - s));
    } else {
        uint64_t mag = (uint64_t)(D < 0 ? -D : D) << (63 - s);
        uint64_t q = (uint64_t)(((u128)mag * FX_RJ[j - 45]) >> 64);
        r = D < 0 ? -(int64_t)q : (int64_t)q;
    }
    int64_t t = FX_LOGC[9];
    for (int k = 8; k >= 1; k--) t = FX_LOGC[k] - (int64_t)(((i128)r * t) >> 63);
    i128 sum = (i128)e * FX_LN2 + FX_LNJ[j - 45] + (((i128)r * t) >> 9);
    if (sum == 0) return 0.0;
    return fx_to_double(sum, 116);
}

double orc_det_exp(double x) {
    if (x != x) return NAN;
    if (x > 710.0) return INFINITY;
    if (x < -746.0) return 0.0;
    fx_init();
    double kd = floor(x * 0x1.71547652b82fep+6 + 0.5);
    int k = (int)kd;
    uint64_t bits;
    memcpy(&bits, &x, 8);
    int be = (int)((bits >> 52) & 0x7ff);
    i128 X = 0;
    if (be != 0) {
        uint64_t sig = (bits & 0x000fffffffffffffULL) | 0x0010000000000000ULL;
        int sh = be - 1075 + 116;
        u128 mag;
        if (sh >= 0)
            mag = (u128)sig << sh;
        else if (sh > -64)
            mag = (u128)(sig >> (-sh));
        else
            mag = 0;
        X = (bits >> 63) ? -(i128)mag : (i128)mag;
    }
    i128 R = X - (i128)k * FX_LN2_64;
    int64_t r = (int64_t)(R >> 54);
    int64_t p = FX_EXPC[7];
    for (int i = 6; i >= 0; i--) p = FX_EXPC[i] + (int64_t)(((i128)r * p) >> 62);
    int j = k & 63;
    int m = (k - j) / 64;
    uint64_t v62 = (uint64_t)(((u128)(uint64_t)p * FX_E2[j]) >> 62);
    double v = fx_to_double((i128)v62, 62);
    if (m > 1023) return (v * pow2i(1023)) * pow2i(m - 1023);
    if (m < -1021) return (v * pow2i(m + 600)) * pow2i(-600);
    return v * pow2i(m);
}

/* ln(1+x) for x > -1; for |x| < 1/4 via 2 atanh(x/(2+x)), else det_log(1+x). */
double orc_det_log1p(double x) {
    if (x != x || x < -1.0) return NAN;
    if (x == -1.0) return -INFINITY;
    if (x < -0.25 || x > 0.25) return orc_det_log(1.0 + x);
    double s = x / (2.0 + x);
    return two_atanh_series(s);
}


double orc_det_pow(double x, double y) { return orc_det_exp(y * orc_det_log(x)); }

/* sin(pi x) for x in [0, 1/2]: Taylor series of sin or of cos(pi (1/2 - x)). */
double orc_det_sinpi(double x) {
    if (x <= 0.25) {
        double y = x * PI_D;
        double z = y * y;
        double p = -1.0 / 1307674368000.0;    /* -1/15! */
        p = 1.0 / 6227020800.0 + z * p;       /* 1/13! */
        p = -1.0 / 39916800.0 + z * p;        /* -1/11! */
        p = 1.0 / 362880.0 + z * p;           /* 1/9! */
        p = -1.0 / 5040.0 + z * p;            /* -1/7! */
        p = 1.0 / 120.0 + z * p;              /* 1/5! */
        p = -1.0 / 6.0 + z * p;               /* -1/3! */
        double t = y * z;
        return y + t * p;
    }
    double y = (0.5 - x) * PI_D;
    double z = y * y;
    double p = 1.0 / 20922789888000.0;   /* 1/16! */
    p = -1.0 / 87178291200.0 + z * p;    /* -1/14! */
    p = 1.0 / 479001600.0 + z * p;       /* 1/12! */
    p = -1.0 / 3628800.0 + z * p;        /* -1/10! */
    p = 1.0 / 40320.0 + z * p;           /* 1/8! */
    p = -1.0 / 720.0 + z * p;            /* -1/6! */
    p = 1.0 / 24.0 + z * p;              /* 1/4! */
    p = -0.5 + z * p;                    /* -1/2! */
    return 1.0 + z * p;
}

/* acosh z = ln(z + sqrt(z^2 - 1)), z >= 1. */
double orc_det_acosh(double z) { return orc_det_log(z + sqrt(z * z - 1.0)); }
#endif /* ORC_PLAIN */

/* x^(1/d) for the threshold variant; x for d = 1. */
static double root_d(double x, int d) {
    if (d == 1) return x;
    return orc_det_exp(orc_det_log(x) / (double)d);
}

/* ------------------------------------------------------------------------ */
/* Exact sum of positive doubles (W = sum of weights, Sec. 2.1)               */
/* ------------------------------------------------------------------------ */

/* Exact fixed-point accumulation in 128-bit integers, then one
 * round-to-nearest-even conversion.  Returns -1 if the dynamic range does not
 * fit 128 bits. */
double orc_exact_sum(int64_t n, const double* w) {
    if (n <= 0) return 0.0;
    double wmin = w[0];
    for (int64_t v = 1; v < n; v++)
        if (w[v] < wmin) wmin = w[v];
    int emin;
    frexp(wmin, &emin);
    int E0 = emin - 53; /* every weight is an integer multiple of 2^E0 */
    unsigned __int128 acc = 0;
    for (int64_t v = 0; v < n; v++) {
        double scaled = ldexp(w[v], -E0);
        if (scaled >= 0x1p120) return -1.0;
        unsigned __int128 m = (unsigned __int128)scaled;
        unsigned __int128 before = acc;
        acc += m;
        if (acc < before) return -1.0;
    }
    /* round acc to 53 significant bits, ties to even */
    int top = 127;
    while (top >= 0 && !((acc >> top) & 1)) top--;
    if (top < 53) return ldexp((double)(uint64_t)acc, E0);
    int shift = top - 52;
    unsigned __int128 mant = acc >> shift;
    unsigned __int128 rem = acc & ((((unsigned __int128)1) << shift) - 1);
    unsigned __int128 half = ((unsigned __int128)1) << (shift - 1);
    if (rem > half || (rem == half && (mant & 1))) mant += 1;
    return ldexp((double)(uint64_t)mant, shift + E0);
}

/* ------------------------------------------------------------------------ */
/* Model inputs (Sec. 2.1, Sec. 2.2, Sec. 5.1 steps 1-2)                      */
/* ------------------------------------------------------------------------ */

/* Pareto weights by inversion and uniform fixed-point torus positions;
 * X is row-major [n][d]. */
void orc_girg_points(int64_t n, int d, double beta, double w_min, uint64_t seed, double* w,
                     uint32_t* X) {
    double expo = -1.0 / (beta - 1.0);
    uint32_t o[4];
    for (int64_t v = 0; v < n; v++) {
        uint32_t vlo = (uint32_t)v, vhi = (uint32_t)((uint64_t)v >> 32);
        philox_seed(seed, vlo, vhi, TAG_WEIGHT, 0, o);
        double U = orc_uniform(o[0], o[1]);
        w[v] = w_min * orc_det_pow(U, expo);
        for (int k = 0; k < d; k++) {
            if ((k & 3) == 0) philox_seed(seed, vlo, vhi, TAG_POS, (uint32_t)(k >> 2), o);
            X[v * d + k] = o[k & 3];
        }
    }
}

/* HRG points: radius density alpha sinh(alpha r)/(cosh(alpha R) - 1) by
 * inversion of its CDF (cosh(alpha r) - 1)/(cosh(alpha R) - 1); the angle is
 * theta = 2 pi X 2^-32 with X the fixed-point torus coordinate. */
void orc_hrg_points(int64_t n, double alpha, double R, uint64_t seed, double* r, uint32_t* X) {
    double ea = orc_det_exp(alpha * R);
    double cosh_aR = (ea + 1.0 / ea) * 0.5;
    uint32_t o[4];
    for (int64_t v = 0; v < n; v++) {
        uint32_t vlo = (uint32_t)v, vhi = (uint32_t)((uint64_t)v >> 32);
        philox_seed(seed, vlo, vhi, TAG_RADIUS, 0, o);
        double U = orc_uniform(o[0], o[1]);
        r[v] = orc_det_acosh(1.0 + U * (cosh_aR - 1.0)) / alpha;
        philox_seed(seed, vlo, vhi, TAG_POS, 0, o);
        X[v] = o[0];
    }
}

/* HRG -> GIRG mapping (Sec. 2.3): w = e^((R - r)/2); x = theta / 2 pi. */
double orc_hrg_weight(double r, double R) { return orc_det_exp((R - r) * 0.5); }

/* ------------------------------------------------------------------------ */
/* Connection probabilities                                                   */
/* ------------------------------------------------------------------------ */

static uint32_t circ_diff(uint32_t a, uint32_t b) {
    uint32_t t = a - b;
    uint32_t u = b - a;
    return t < u ? t : u;
}

/* L_inf torus distance in units of 2^-32 (Sec. 2.1). */
static uint32_t torus_dist(const uint32_t* xu, const uint32_t* xv, int d) {
    uint32_t m = 0;
    for (int k = 0; k < d; k++) {
        uint32_t t = circ_diff(xu[k], xv[k]);
        if (t > m) m = t;
    }
    return m;
}

/* The GIRG model with its scale K: K = c^T for T > 0 and K = c^d for T = 0,
 * c the constant of Eq. 1.  Eq. 1 reads p = min{1, (K q / r^d)^(1/T)} with
 * q = w_u w_v / W, and the threshold variant connects iff r^d <= K q.  K stays
 * a moderate number for every T, where c = K^(1/T) leaves the range of doubles
 * as T -> 0. */
typedef struct {
    int d;
    double T, K, W;
    int m_int;   /* 1/T when it is an integer in [1,64], else 0 */
    double invT; /* 1/T */
} girg_model;

static void girg_model_init(girg_model* M, int d, double T, double K, double W) {
    M->d = d;
    M->T = T;
    M->K = K;
    M->W = W;
    M->invT = T > 0.0 ? 1.0 / T : 0.0;
    M->m_int = 0;
    if (T > 0.0 && M->invT == floor(M->invT) && M->invT <= 64.0) M->m_int = (int)M->invT;
}

/* Eq. 1 at distance r: x = K q / r^d, p = 1 if x >= 1 else x^(1/T) (repeated
 * products when 1/T is an integer). */
static double girg_p_at(const girg_model* M, double wu, double wv, double r) {
    double q = (wu * wv) / M->W;
    double rd = r;
    for (int k = 1; k < M->d; k++) rd = rd * r;
    double x = (M->K * q) / rd;
    if (x >= 1.0) return 1.0;
    double p;
    if (M->m_int > 0) {
        p = x;
        for (int k = 1; k < M->m_int; k++) p = p * x;
    } else {
        p = orc_det_exp(M->invT * orc_det_log(x));
    }
    return p;
}

/* Eq. 1 at the fixed-point distance D (r = D 2^-32; r = 0 gives p = 1). */
static double girg_p(const girg_model* M, double wu, double wv, uint32_t D) {
    if (D == 0) return 1.0;
    return girg_p_at(M, wu, wv, (double)D * 0x1p-32);
}

/* The two sides of the threshold variant's test: r^d and K w_u w_v / W. */
static void girg_thresh_sides(const girg_model* M, double wu, double wv, uint32_t D, double* rd,
                              double* kq) {
    double q = (wu * wv) / M->W;
    double r = (double)D * 0x1p-32;
    double x = r;
    for (int k = 1; k < M->d; k++) x = x * r;
    *rd = x;
    *kq = M->K * q;
}

/* Threshold variant: edge iff ||x_u - x_v||^d <= K w_u w_v / W (r <= c q^(1/d)). */
static int girg_thresh_edge(const girg_model* M, double wu, double wv, uint32_t D) {
    double rd, kq;
    girg_thresh_sides(M, wu, wv, D, &rd, &kq);
    return rd <= kq;
}

/* K from the c of Eq. 1: c^T (T > 0) or c^d (T = 0). */
double orc_girg_K_of_c(double c, int d, double T) {
    if (T > 0.0) return orc_det_pow(c, T);
    double k = c;
    for (int i = 1; i < d; i++) k = k * c;
    return k;
}

double orc_girg_p(int d, double T, double K, double W, double wu, double wv, uint32_t D) {
    girg_model M;
    girg_model_init(&M, d, T, K, W);
    return girg_p(&M, wu, wv, D);
}

int orc_girg_thresh_edge(int d, double K, double W, double wu, double wv, uint32_t D) {
    girg_model M;
    girg_model_init(&M, d, 0.0, K, W);
    return girg_thresh_edge(&M, wu, wv, D);
}

typedef struct {
    double T, R;
    double coshR;
} hrg_model;

static void hrg_model_init(hrg_model* H, double T, double R) {
    H->T = T;
    H->R = R;
    double eR = orc_det_exp(R);
    H->coshR = (eR + 1.0 / eR) * 0.5;
}

/* cosh of the hyperbolic distance (Sec. 2.2) in the form
 * cosh(r_u - r_v) + 2 sinh r_u sinh r_v sin^2(dtheta / 2),
 * with E = e^r, sh = sinh r per vertex and dtheta / 2 = pi D 2^-32. */
static double hrg_coshd(double Eu, double shu, double Ev, double shv, uint32_t D) {
    double s = orc_det_sinpi((double)D * 0x1p-32);
    double ch = (Eu / Ev + Ev / Eu) * 0.5;
    double t = shu * shv;
    t = t * (s * s);
    return ch + 2.0 * t;
}

/* p_T(d) = 1 / (exp((d - R) / 2T) + 1), d = acosh(cosh d). */
static double hrg_p_from_coshd(const hrg_model* H, double coshd) {
    double dist = orc_det_acosh(coshd);
    return 1.0 / (orc_det_exp((dist - H->R) / (2.0 * H->T)) + 1.0);
}

double orc_hrg_coshd(double ru, double rv, uint32_t D) {
    double Eu = orc_det_exp(ru), Ev = orc_det_exp(rv);
    double shu = (Eu - 1.0 / Eu) * 0.5, shv = (Ev - 1.0 / Ev) * 0.5;
    return hrg_coshd(Eu, shu, Ev, shv, D);
}

double orc_hrg_p(double T, double R, double ru, double rv, uint32_t D) {
    hrg_model H;
    hrg_model_init(&H, T, R);
    double cd = orc_hrg_coshd(ru, rv, D);
    if (T == 0.0) return cd < H.coshR ? 1.0 : 0.0;
    return hrg_p_from_coshd(&H, cd);
}

/* ------------------------------------------------------------------------ */
/* Oracle 1: all pairs (Table 1 "Pairwise"), edge iff U(seed,u,v) < p_uv.     */
/* ------------------------------------------------------------------------ */

static double pair_coin(uint64_t seed, uint32_t u, uint32_t v) {
    uint32_t o[4];
    philox_seed(seed, u, v, TAG_PAIR, 0, o);
    return orc_uniform(o[0], o[1]);
}

double orc_pair_coin(uint64_t seed, uint32_t u, uint32_t v) { return pair_coin(seed, u, v); }

/* Decision audit (a test aid; off unless orc_audit_begin was called).  It changes no
 * decision: it counts every decision the samplers take and records those whose two
 * sides are within a relative eps of each other, the only ones that a different
 * rounding of the same formulas can flip.  A record is three int64 (kind, a, b):
 *   kind 1  per-pair coin U < p (a < b vertex ids),
 *   kind 2  type-II acceptance U' pbar < p (a < b vertex ids),
 *   kind 3  threshold test r^d <= K q (GIRG) or cosh d < cosh R (HRG) (a < b ids),
 *   kind 4  geometric jump whose quotient ln U / ln(1 - pbar) lies within a relative
 *           eps of an integer (a = cell A, b = stream word << 32 | chunk). */
static struct {
    int on;
    double eps;
    int64_t* buf;
    int64_t cap, n, decisions;
} g_audit;

void orc_audit_begin(double eps, int64_t* buf, int64_t cap) {
    g_audit.on = 1;
    g_audit.eps = eps;
    g_audit.buf = buf;
    g_audit.cap = cap;
    g_audit.n = 0;
    g_audit.decisions = 0;
}

/* Stops the audit; returns the number of records (more than cap: only cap stored). */
int64_t orc_audit_end(int64_t* decisions) {
    if (decisions) *decisions = g_audit.decisions;
    g_audit.on = 0;
    return g_audit.n;
}

static void audit_record(int64_t kind, int64_t a, int64_t b) {
    if (g_audit.n < g_audit.cap) {
        g_audit.buf[3 * g_audit.n] = kind;
        g_audit.buf[3 * g_audit.n + 1] = a;
        g_audit.buf[3 * g_audit.n + 2] = b;
    }
    g_audit.n++;
}

/* One decision between x and y (x < y or x <= y): recorded when |x - y| <= eps |y|. */
static void audit_cmp(int kind, double x, double y, int64_t a, int64_t b) {
    if (!g_audit.on) return;
    g_audit.decisions++;
    if (fabs(x - y) <= g_audit.eps * fabs(y)) audit_record(kind, a, b);
}

static void emit(uint32_t* edges, int64_t cap, int64_t* m, uint32_t a, uint32_t b) {
    if (a > b) {
        uint32_t t = a;
        a = b;
        b = t;
    }
    if (*m < cap) {
        edges[2 * *m] = a;
        edges[2 * *m + 1] = b;
    }
    (*m)++;
}

int64_t orc_girg_allpairs(int64_t n, int d, const uint32_t* X, const double* w, double W,
                          double T, double K, uint64_t seed, uint32_t* edges, int64_t cap) {
    girg_model M;
    girg_model_init(&M, d, T, K, W);
    int64_t m = 0;
    for (int64_t u = 0; u < n; u++) {
        for (int64_t v = u + 1; v < n; v++) {
            uint32_t D = torus_dist(X + u * d, X + v * d, d);
            int e;
            if (T == 0.0) {
                double rd, kq;
                girg_thresh_sides(&M, w[u], w[v], D, &rd, &kq);
                audit_cmp(3, rd, kq, u, v);
                e = rd <= kq;
            } else {
                double U = pair_coin(seed, (uint32_t)u, (uint32_t)v), p = girg_p(&M, w[u], w[v], D);
                audit_cmp(1, U, p, u, v);
                e = U < p;
            }
            if (e) emit(edges, cap, &m, (uint32_t)u, (uint32_t)v);
        }
    }
    return m;
}

int64_t orc_hrg_allpairs(int64_t n, const uint32_t* X, const double* r, double R, double T,
                         uint64_t seed, uint32_t* edges, int64_t cap) {
    hrg_model H;
    hrg_model_init(&H, T, R);
    double* E = malloc(sizeof(double) * (n ? n : 1));
    double* sh = malloc(sizeof(double) * (n ? n : 1));
    for (int64_t v = 0; v < n; v++) {
        E[v] = orc_det_exp(r[v]);
        sh[v] = (E[v] - 1.0 / E[v]) * 0.5;
    }
    int64_t m = 0;
    for (int64_t u = 0; u < n; u++) {
        for (int64_t v = u + 1; v < n; v++) {
            uint32_t D = circ_diff(X[u], X[v]);
            double cd = hrg_coshd(E[u], sh[u], E[v], sh[v], D);
            int e;
            if (T == 0.0) {
                audit_cmp(3, cd, H.coshR, u, v);
                e = cd < H.coshR;
            } else {
                double U = pair_coin(seed, (uint32_t)u, (uint32_t)v), p = hrg_p_from_coshd(&H, cd);
                audit_cmp(1, U, p, u, v);
                e = U < p;
            }
            if (e) emit(edges, cap, &m, (uint32_t)u, (uint32_t)v);
        }
    }
    free(E);
    free(sh);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Oracle 2: the cell-pair sampler (Algorithm 1 with App. B.1)               */
/* ------------------------------------------------------------------------ */

/* Morton code of the cell containing x at level l: bit b of coordinate k
 * lands at position b*d + (d-1-k), so coordinate 0 is the most significant
 * bit of every d-bit group (Sec. 4.2: a3 b3 a2 b2 a1 b1 a0 b0). */
uint64_t orc_morton(const uint32_t* x, int d, int l) {
    uint64_t code = 0;
    for (int b = 0; b < l; b++) {
        for (int k = 0; k < d; k++) {
            uint32_t coord = x[k] >> (32 - l);
            uint64_t bit = (coord >> b) & 1u;
            code |= bit << (b * d + (d - 1 - k));
        }
    }
    return code;
}

/* Coordinates of a cell from its Morton code. */
static void morton_decode(uint64_t code, int d, int l, uint32_t* coord) {
    for (int k = 0; k < d; k++) coord[k] = 0;
    for (int b = 0; b < l; b++)
        for (int k = 0; k < d; k++) coord[k] |= (uint32_t)((code >> (b * d + (d - 1 - k))) & 1u) << b;
}

/* Largest per-dimension circular difference between the cells (their
 * L_inf cell distance); cells are neighbours iff it is <= 1 (a cell is its
 * own neighbour; on levels 0 and 1 all cells are neighbours). */
static uint32_t cell_linf(uint64_t A, uint64_t B, int d, int l) {
    uint32_t ca[MAXD], cb[MAXD];
    morton_decode(A, d, l, ca);
    morton_decode(B, d, l, cb);
    uint32_t side = l >= 32 ? 0u : (1u << l);
    uint32_t m = 0;
    for (int k = 0; k < d; k++) {
        uint32_t diff = ca[k] > cb[k] ? ca[k] - cb[k] : cb[k] - ca[k];
        uint32_t wrap = side - diff;
        if (wrap < diff) diff = wrap;
        if (diff > m) m = diff;
    }
    return m;
}

uint32_t orc_cell_linf(uint64_t A, uint64_t B, int d, int l) { return cell_linf(A, B, d, l); }

/* Deepest level used (the paper leaves the maximum depth open).  Capping a
 * comparison level only makes cells coarser; the sample stays exact because every
 * bound is computed from the actual cells.  Levels beyond floor(32/d) have no room
 * in a 32-bit Morton code.  At T = 0 there are no distant items, and levels with
 * more than 2^(bitlen(n)+4) <= 32 n cells gain nothing.  At T > 0 a cell with m
 * vertices of a bucket costs about 3^d m^2 type-I pair tests and 6^d - 3^d distant
 * partner cells; with N cells and n vertices the sum 3^d n^2 / N + (6^d - 3^d) N is
 * smallest near N = n 2^(-d/2), i.e. at the level floor(log2(n) / d - 1/2), with
 * log2 n taken as bitlen(n) - 1. */
int orc_level_cap(int64_t n, int d, double T) {
    int bitlen = 0;
    while (bitlen < 63 && ((int64_t)1 << bitlen) <= n) bitlen++;
    int a = 32 / d;
    int b = T > 0.0 ? (2 * bitlen - 2 - d) / (2 * d) : (bitlen + 4) / d;
    if (b < 1) b = 1;
    return a < b ? a : b;
}

/* Largest level l in [0, cap] with cell side 2^-l > kappa (1 + 2^-30),
 * i.e. the comparison level of Sec. 3.1 for the threshold distance kappa. */
static int level_for_kappa(double kappa, int cap) {
    double k2 = kappa * (1.0 + 0x1p-30);
    int l = 0;
    while (l < cap && ldexp(1.0, -(l + 1)) > k2) l++;
    return l;
}

/* Chunk length exponent for geometric jumps under bound pbar: 2^k pbar in
 * [4, 8) when not clamped to [3, 31]. */
int orc_chunk_log(double pbar) {
    int e;
    frexp(pbar, &e);
    int k = 3 - e;
    if (k < 3) k = 3;
    if (k > 31) k = 31;
    return k;
}

/* A type-II item (cell pair, bucket pair) awaiting its stream: V_i^A x V_j^B at
 * level l with gap g; rank orders B among the partners of A (t2_rank). */
struct t2rec {
    uint32_t A, B;
    uint8_t l, i, j, g;
    uint32_t rank;
};

typedef struct {
    int model; /* 0 GIRG, 1 HRG */
    int64_t n;
    int d;
    uint64_t seed;
    const uint32_t* X;
    const double* w; /* GIRG weights, or HRG mapped weights */
    girg_model M;
    hrg_model H;
    const double* r; /* HRG radii */
    double* E;       /* HRG e^r */
    double* sh;      /* HRG sinh r */
    /* buckets and levels */
    int L;
    int64_t lcount[MAXL];
    double wmax[MAXL];
    double rlo[MAXL], rhi[MAXL];
    int CL[MAXL][MAXL];
    int I[MAXL];
    int Dmax;
    int lcap;
    int64_t* order;       /* sorted position -> vertex id */
    int64_t lstart[MAXL + 1];
    int64_t* offs[MAXL];  /* per layer: 2^(d I(i)) + 1 prefix sums */
    /* output */
    uint32_t* edges;
    int64_t cap;
    int64_t m;
    /* statistics: [0] type-I pairs tested, [1] type-II items, [2] jump draws,
     * [3] type-II candidates, [4] type-I items, [5] cell pairs visited,
     * [6] type-I edges, [7] type-II edges */
    int64_t stats[8];
    /* visited cell pairs per level: neighbours, distant, and (A, A) pairs */
    int64_t lvl_nb[33], lvl_far[33], lvl_self[33];
    /* type-II items collected by the recursion, sampled per stream afterwards */
    struct t2rec* t2;
    int64_t n_t2, cap_t2;
    int64_t error;
    /* optional item log: 12 int64 per item */
    int64_t* items;
    int64_t items_cap;
    int64_t n_items;
    int skip_sampling;
} cp_ctx;

static int layer_of(double w, double w_min) {
    int e;
    frexp(w / w_min, &e); /* w / w_min = m 2^e, m in [0.5, 1) */
    int layer = e - 1;
    if (layer < 0) layer = 0;
    if (layer > MAXL - 1) layer = MAXL - 1;
    return layer;
}

/* The weight bucket of Sec. 3.1 (exported for its tests). */
int orc_layer_of(double w, double w_min) { return layer_of(w, w_min); }

/* Sorting key: (bucket, Morton code of the insertion-level cell, id). */
typedef struct {
    int layer;
    uint64_t cell;
    int64_t id;
} sort_rec;

static int cmp_rec(const void* a, const void* b) {
    const sort_rec* x = a;
    const sort_rec* y = b;
    if (x->layer != y->layer) return x->layer < y->layer ? -1 : 1;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/* Comparison level of a bucket pair, Sec. 3.1 (GIRG: closed form of the
 * threshold distance at the largest weights; HRG: level search, Sec. 4.3). */
static int comparison_level(cp_ctx* C, int i, int j) {
    if (C->model == 0) {
        const girg_model* M = &C->M;
        double qmax = (C->wmax[i] * C->wmax[j]) / M->W;
        /* the distance at which p reaches 1 (T > 0) or the threshold (T = 0) */
        double kappa = root_d(M->K * qmax, M->d);
        return level_for_kappa(kappa, C->lcap);
    }
    /* HRG: deepest level whose distant cell pairs (angular gap >= one cell)
     * cannot hold a threshold edge, by the lower bound on cosh d. */
    double gap = 0.0;
    if (C->rlo[j] > C->rhi[i]) gap = C->rlo[j] - C->rhi[i];
    if (C->rlo[i] > C->rhi[j]) gap = C->rlo[i] - C->rhi[j];
    double eg = orc_det_exp(gap);
    double cg = (eg + 1.0 / eg) * 0.5;
    double ei = orc_det_exp(C->rlo[i]), ej = orc_det_exp(C->rlo[j]);
    double shi = (ei - 1.0 / ei) * 0.5, shj = (ej - 1.0 / ej) * 0.5;
    double limit = C->H.coshR * (1.0 + 0x1p-30);
    int l = 1;
    while (l < C->lcap) {
        double s = orc_det_sinpi(ldexp(1.0, -(l + 1)));
        double t = shi * shj;
        t = t * (s * s);
        double lb = cg + 2.0 * t;
        if (!(lb > limit)) break;
        l++;
    }
    return l;
}

/* Upper bound on p over a distant item at level l whose cells are g cells
 * apart (Sec. 3.2: largest weights of the buckets, smallest distance of the
 * cells), inflated by 2^-30 and clamped to 1. */
static double type2_bound(cp_ctx* C, int i, int j, int l, uint32_t g) {
    double p;
    if (C->model == 0) {
        double rmin = (double)g * ldexp(1.0, -l);
        p = girg_p_at(&C->M, C->wmax[i], C->wmax[j], rmin);
    } else {
        double gap = 0.0;
        if (C->rlo[j] > C->rhi[i]) gap = C->rlo[j] - C->rhi[i];
        if (C->rlo[i] > C->rhi[j]) gap = C->rlo[i] - C->rhi[j];
        double eg = orc_det_exp(gap);
        double cg = (eg + 1.0 / eg) * 0.5;
        double ei = orc_det_exp(C->rlo[i]), ej = orc_det_exp(C->rlo[j]);
        double shi = (ei - 1.0 / ei) * 0.5, shj = (ej - 1.0 / ej) * 0.5;
        double s = orc_det_sinpi((double)g * ldexp(1.0, -l));
        double t = shi * shj;
        t = t * (s * s);
        double lb = cg + 2.0 * t;
        p = hrg_p_from_coshd(&C->H, lb);
    }
    p = p * (1.0 + 0x1p-30);
    return p < 1.0 ? p : 1.0;
}

/* Does the pair of vertices (ids) form an edge under the per-pair coin? */
static int type1_decide(cp_ctx* C, int64_t u, int64_t v) {
    uint32_t a = (uint32_t)(u < v ? u : v), b = (uint32_t)(u < v ? v : u);
    if (C->model == 0) {
        uint32_t D = torus_dist(C->X + (int64_t)a * C->d, C->X + (int64_t)b * C->d, C->d);
        if (C->M.T == 0.0) {
            double rd, kq;
            girg_thresh_sides(&C->M, C->w[a], C->w[b], D, &rd, &kq);
            audit_cmp(3, rd, kq, a, b);
            return rd <= kq;
        }
        double U = pair_coin(C->seed, a, b), p = girg_p(&C->M, C->w[a], C->w[b], D);
        audit_cmp(1, U, p, a, b);
        return U < p;
    }
    uint32_t D = circ_diff(C->X[a], C->X[b]);
    double cd = hrg_coshd(C->E[a], C->sh[a], C->E[b], C->sh[b], D);
    if (C->H.T == 0.0) {
        audit_cmp(3, cd, C->H.coshR, a, b);
        return cd < C->H.coshR;
    }
    double U = pair_coin(C->seed, a, b), p = hrg_p_from_coshd(&C->H, cd);
    audit_cmp(1, U, p, a, b);
    return U < p;
}

static double pair_p(cp_ctx* C, int64_t u, int64_t v) {
    uint32_t a = (uint32_t)(u < v ? u : v), b = (uint32_t)(u < v ? v : u);
    if (C->model == 0) {
        uint32_t D = torus_dist(C->X + (int64_t)a * C->d, C->X + (int64_t)b * C->d, C->d);
        return girg_p(&C->M, C->w[a], C->w[b], D);
    }
    uint32_t D = circ_diff(C->X[a], C->X[b]);
    double cd = hrg_coshd(C->E[a], C->sh[a], C->E[b], C->sh[b], D);
    return hrg_p_from_coshd(&C->H, cd);
}

/* V_i^A as a range of sorted positions, for level(A) = l <= I(i) (Lemma 1). */
static void vrange(cp_ctx* C, int i, uint64_t A, int l, int64_t* lo, int64_t* hi) {
    int s = C->d * (C->I[i] - l);
    *lo = C->lstart[i] + C->offs[i][A << s];
    *hi = C->lstart[i] + C->offs[i][(A + 1) << s];
}

static void log_item(cp_ctx* C, int type, int l, uint64_t A, uint64_t B, int i, int j,
                     int64_t alo, int64_t ahi, int64_t blo, int64_t bhi, int tri, double pbar) {
    if (!C->items) return;
    if (C->n_items < C->items_cap) {
        int64_t* it = C->items + 12 * C->n_items;
        it[0] = type;
        it[1] = l;
        it[2] = (int64_t)A;
        it[3] = (int64_t)B;
        it[4] = i;
        it[5] = j;
        it[6] = alo;
        it[7] = ahi;
        it[8] = blo;
        it[9] = bhi;
        it[10] = tri;
        memcpy(&it[11], &pbar, 8);
    }
    C->n_items++;
}

/* Type I (Algorithm 1, line 3): every pair of V_i^A x V_j^B; when the item
 * is (A, A, i, i) only pairs at sorted positions a < b (App. B.1). */
static void type1_item(cp_ctx* C, int l, uint64_t A, uint64_t B, int i, int j) {
    int64_t alo, ahi, blo, bhi;
    vrange(C, i, A, l, &alo, &ahi);
    vrange(C, j, B, l, &blo, &bhi);
    if (alo == ahi || blo == bhi) return;
    int tri = (A == B && i == j);
    C->stats[4]++;
    log_item(C, 1, l, A, B, i, j, alo, ahi, blo, bhi, tri, 1.0);
    if (C->skip_sampling) return;
    for (int64_t a = alo; a < ahi; a++) {
        for (int64_t b = tri ? a + 1 : blo; b < bhi; b++) {
            C->stats[0]++;
            int64_t u = C->order[a], v = C->order[b];
            if (type1_decide(C, u, v)) {
                emit(C->edges, C->cap, &C->m, (uint32_t)u, (uint32_t)v);
                C->stats[6]++;
            }
        }
    }
}

/* Rank of a distant cell B among the partners of A at level l (>= 2): B is a
 * child of a neighbour P of parent(A); with e_k in {-1, 0, 1} the offset of P
 * from parent(A) in dimension k (on a level of 2 cells per dimension the other
 * cell counts as +1) and kid_k the lowest coordinate bit of B,
 * rank = (sum_k (e_k + 1) 3^(d-1-k)) 2^d + sum_k kid_k 2^(d-1-k). */
static uint32_t t2_rank(uint64_t A, uint64_t B, int d, int l) {
    uint32_t pa[MAXD], pb[MAXD], cb[MAXD];
    morton_decode(A >> d, d, l - 1, pa);
    morton_decode(B >> d, d, l - 1, pb);
    morton_decode(B, d, l, cb);
    uint32_t side = 1u << (l - 1);
    uint32_t eidx = 0, kids = 0;
    for (int k = 0; k < d; k++) {
        uint32_t diff = (pb[k] - pa[k]) & (side - 1); /* 0, 1 or side - 1 */
        int e = diff == 0 ? 0 : (diff == 1 ? 1 : -1);
        eidx = eidx * 3 + (uint32_t)(e + 1);
        kids = (kids << 1) | (cb[k] & 1u);
    }
    return (eidx << d) | kids;
}

/* Type II (Algorithm 1, lines 5-6): record the item; the candidates are chosen
 * later by geometric jumps per stream (sample_streams). */
static void type2_item(cp_ctx* C, int l, uint64_t A, uint64_t B, int i, int j) {
    int64_t alo, ahi, blo, bhi;
    vrange(C, i, A, l, &alo, &ahi);
    vrange(C, j, B, l, &blo, &bhi);
    if (alo == ahi || blo == bhi) return;
    uint32_t g = cell_linf(A, B, C->d, l) - 1;
    double pbar = type2_bound(C, i, j, l, g);
    C->stats[1]++;
    log_item(C, 2, l, A, B, i, j, alo, ahi, blo, bhi, 0, pbar);
    if (C->skip_sampling) return;
    if (C->n_t2 == C->cap_t2) {
        C->cap_t2 = C->cap_t2 ? 2 * C->cap_t2 : 1 << 16;
        C->t2 = realloc(C->t2, sizeof(struct t2rec) * (size_t)C->cap_t2);
    }
    struct t2rec* r = &C->t2[C->n_t2++];
    r->A = (uint32_t)A;
    r->B = (uint32_t)B;
    r->l = (uint8_t)l;
    r->i = (uint8_t)i;
    r->j = (uint8_t)j;
    r->g = (uint8_t)g;
    r->rank = t2_rank(A, B, C->d, l);
}

static int cmp_t2(const void* a, const void* b) {
    const struct t2rec* x = a;
    const struct t2rec* y = b;
    if (x->l != y->l) return x->l < y->l ? -1 : 1;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    if (x->j != y->j) return x->j < y->j ? -1 : 1;
    if (x->A != y->A) return x->A < y->A ? -1 : 1;
    if (x->g != y->g) return x->g < y->g ? -1 : 1;
    if (x->rank != y->rank) return x->rank < y->rank ? -1 : 1;
    return 0;
}

/* One geometric jump (Sec. 3.2) under a bound pbar < 1, Lb = ln(1 - pbar), from the
 * uniform U of the words (lo, hi): X = floor(ln U / Lb), the number of positions skipped
 * before the next candidate; -1 where X >= 2^63 (the stream then leaves its chunk). */
static double jump_quotient(double Lb, uint32_t lo, uint32_t hi) {
    return orc_det_log(orc_uniform(lo, hi)) / Lb;
}

static int64_t geometric_jump(double Lb, uint32_t lo, uint32_t hi) {
    double x = floor(jump_quotient(Lb, lo, hi));
    return x >= 0x1p63 ? -1 : (int64_t)x;
}

/* The jumps under a bound pbar in (0, 1) for n word pairs (the tests check their law). */
void orc_geometric_jumps(int64_t n, double pbar, const uint32_t* lo, const uint32_t* hi,
                         int64_t* out) {
    double Lb = orc_det_log1p(-pbar);
    for (int64_t q = 0; q < n; q++) out[q] = geometric_jump(Lb, lo[q], hi[q]);
}

/* Geometric jumps (Sec. 3.2) with the bound pbar over the index space
 * idx = a S + b of V_i^A x (V_j^B1 ++ V_j^B2 ++ ...), S the total size of the
 * stream's partner sets, cut into chunks of 2^k indices; a candidate is
 * accepted with probability p_uv / pbar, as U' pbar < p_uv. */
static void sample_stream(cp_ctx* C, const struct t2rec* m, int64_t nm) {
    int l = m[0].l, i = m[0].i, j = m[0].j;
    uint32_t g = m[0].g;
    uint64_t A = m[0].A;
    int64_t alo, ahi;
    vrange(C, i, A, l, &alo, &ahi);
    int64_t* blo = malloc(sizeof(int64_t) * (size_t)nm);
    uint64_t* pre = malloc(sizeof(uint64_t) * (size_t)(nm + 1));
    pre[0] = 0;
    for (int64_t q = 0; q < nm; q++) {
        int64_t lo, hi;
        vrange(C, j, m[q].B, l, &lo, &hi);
        blo[q] = lo;
        pre[q + 1] = pre[q] + (uint64_t)(hi - lo);
    }
    uint64_t na = (uint64_t)(ahi - alo), S = pre[nm];
    uint64_t total = na * S;
    double pbar = type2_bound(C, i, j, l, g);
    int k = orc_chunk_log(pbar);
    uint64_t chunk = (uint64_t)1 << k;
    uint64_t nchunks = (total + chunk - 1) >> k;
    if (nchunks > 0xffffffffULL) C->error = 1;
    double Lb = pbar < 1.0 ? orc_det_log1p(-pbar) : 0.0;
    uint32_t pack = (uint32_t)l | ((uint32_t)i << 5) | ((uint32_t)j << 11) | ((g - 1) << 17) |
                    (TAG_JUMP << 18);
    for (uint64_t h = 0; h < nchunks && h <= 0xffffffffULL; h++) {
        uint64_t start = h << k;
        uint64_t len = total - start < chunk ? total - start : chunk;
        int64_t s = -1; /* offset of the last candidate within the chunk */
        for (uint32_t t = 0;; t++) {
            uint32_t o[4];
            philox_seed(C->seed, (uint32_t)A, pack, (uint32_t)h, t, o);
            C->stats[2]++;
            /* stop when the jump leaves the chunk */
            uint64_t remaining = len - (uint64_t)(s + 1);
            uint64_t X = 0;
            if (pbar < 1.0) {
                int64_t x = geometric_jump(Lb, o[0], o[1]);
                if (g_audit.on) { /* distance of the quotient from its nearest integer */
                    double xq = jump_quotient(Lb, o[0], o[1]), k = floor(xq + 0.5);
                    g_audit.decisions++;
                    if (k >= 1.0 && fabs(xq - k) <= g_audit.eps * k)
                        audit_record(4, (int64_t)A, ((int64_t)pack << 32) | (int64_t)h);
                }
                if (x < 0) break;
                X = (uint64_t)x;
            }
            if (X >= remaining) break;
            s = s + 1 + (int64_t)X;
            uint64_t idx = start + (uint64_t)s;
            uint64_t ib = idx % S;
            int64_t q = 0; /* partner set holding position ib */
            while (pre[q + 1] <= ib) q++;
            int64_t u = C->order[alo + (int64_t)(idx / S)];
            int64_t v = C->order[blo[q] + (int64_t)(ib - pre[q])];
            C->stats[3]++;
            double acc = orc_uniform(o[2], o[3]) * pbar, p = pair_p(C, u, v);
            audit_cmp(2, acc, p, u < v ? u : v, u < v ? v : u);
            if (acc < p) {
                emit(C->edges, C->cap, &C->m, (uint32_t)u, (uint32_t)v);
                C->stats[7]++;
            }
        }
    }
    free(blo);
    free(pre);
}

/* Group the recorded type-II items into streams (same l, i, j, A and gap g),
 * partners in increasing rank, and sample each stream. */
static void sample_streams(cp_ctx* C) {
    if (C->n_t2 == 0) return;
    qsort(C->t2, (size_t)C->n_t2, sizeof(struct t2rec), cmp_t2);
    int64_t q0 = 0;
    while (q0 < C->n_t2) {
        int64_t q1 = q0 + 1;
        while (q1 < C->n_t2 && C->t2[q1].l == C->t2[q0].l && C->t2[q1].i == C->t2[q0].i &&
               C->t2[q1].j == C->t2[q0].j && C->t2[q1].A == C->t2[q0].A &&
               C->t2[q1].g == C->t2[q0].g)
            q1++;
        sample_stream(C, C->t2 + q0, q1 - q0);
        q0 = q1;
    }
}

/* Process the cell pair {A, B} (A <= B) at level l for every bucket pair,
 * then recurse into the children while A and B are neighbours
 * (Algorithm 1).  Bucket pairs are taken with i <= j: for A < B and i < j
 * both orientations (A, B) and (B, A) are items, for i = j only (A, B)
 * (App. B.1); type I uses bucket pairs with CL = l, type II those with
 * CL >= l (Sec. 3.3). */
static void recur(cp_ctx* C, int l, uint64_t A, uint64_t B) {
    C->stats[5]++;
    uint32_t linf = cell_linf(A, B, C->d, l);
    int nb = linf <= 1;
    if (nb)
        C->lvl_nb[l]++;
    else
        C->lvl_far[l]++;
    if (A == B) C->lvl_self[l]++;
    for (int i = 0; i < C->L; i++) {
        if (!C->lcount[i]) continue;
        for (int j = i; j < C->L; j++) {
            if (!C->lcount[j]) continue;
            int cl = C->CL[i][j];
            if (nb) {
                if (cl != l) continue;
                type1_item(C, l, A, B, i, j);
                if (A != B && i != j) type1_item(C, l, B, A, i, j);
            } else {
                if (cl < l) continue;
                int thresh = (C->model == 0) ? (C->M.T == 0.0) : (C->H.T == 0.0);
                if (thresh) continue; /* no distant edges at T = 0 (CL margin) */
                type2_item(C, l, A, B, i, j);
                if (i != j) type2_item(C, l, B, A, i, j);
            }
        }
    }
    if (!nb || l >= C->Dmax) return;
    uint64_t nc = (uint64_t)1 << C->d;
    for (uint64_t x = 0; x < nc; x++) {
        for (uint64_t y = (A == B ? x : 0); y < nc; y++) {
            recur(C, l + 1, (A << C->d) | x, (B << C->d) | y);
        }
    }
}

/* Build buckets, levels, the sorted vertex array and the prefix sums
 * (Sec. 3.1, Sec. 3.4, Lemma 1). w_min: the weight unit of the buckets;
 * lcap_override > 0 replaces the default deepest level (a tuning knob that
 * leaves the sample exact). */
static int cp_prepare(cp_ctx* C, double w_min, int lcap_override) {
    int64_t n = C->n;
    int d = C->d;
    C->lcap = orc_level_cap(n, d, C->model == 0 ? C->M.T : C->H.T);
    if (lcap_override > 0) C->lcap = lcap_override < 32 / d ? lcap_override : 32 / d;
    memset(C->lcount, 0, sizeof(C->lcount));
    for (int i = 0; i < MAXL; i++) {
        C->wmax[i] = 0.0;
        C->rlo[i] = INFINITY;
        C->rhi[i] = -INFINITY;
    }
    int* lay = malloc(sizeof(int) * (n ? n : 1));
    C->L = 0;
    for (int64_t v = 0; v < n; v++) {
        int li = layer_of(C->w[v], w_min);
        lay[v] = li;
        C->lcount[li]++;
        if (C->w[v] > C->wmax[li]) C->wmax[li] = C->w[v];
        if (C->model == 1) {
            if (C->r[v] < C->rlo[li]) C->rlo[li] = C->r[v];
            if (C->r[v] > C->rhi[li]) C->rhi[li] = C->r[v];
        }
        if (li + 1 > C->L) C->L = li + 1;
    }
    C->Dmax = 0;
    for (int i = 0; i < C->L; i++) {
        C->I[i] = 0;
        for (int j = 0; j < C->L; j++) C->CL[i][j] = 0;
    }
    for (int i = 0; i < C->L; i++) {
        if (!C->lcount[i]) continue;
        for (int j = i; j < C->L; j++) {
            if (!C->lcount[j]) continue;
            int cl = comparison_level(C, i, j);
            C->CL[i][j] = C->CL[j][i] = cl;
        }
    }
    for (int i = 0; i < C->L; i++) {
        if (!C->lcount[i]) continue;
        for (int j = 0; j < C->L; j++) {
            if (!C->lcount[j]) continue;
            if (C->CL[i][j] > C->I[i]) C->I[i] = C->CL[i][j];
        }
        if (C->I[i] > C->Dmax) C->Dmax = C->I[i];
    }
    sort_rec* rec = malloc(sizeof(sort_rec) * (n ? n : 1));
    for (int64_t v = 0; v < n; v++) {
        rec[v].layer = lay[v];
        rec[v].cell = orc_morton(C->X + v * d, d, C->I[lay[v]]);
        rec[v].id = v;
    }
    qsort(rec, (size_t)n, sizeof(sort_rec), cmp_rec);
    C->order = malloc(sizeof(int64_t) * (n ? n : 1));
    for (int64_t p = 0; p < n; p++) C->order[p] = rec[p].id;
    C->lstart[0] = 0;
    for (int i = 0; i < MAXL; i++) C->lstart[i + 1] = C->lstart[i] + (i < C->L ? C->lcount[i] : 0);
    for (int i = 0; i < MAXL; i++) C->offs[i] = NULL;
    for (int i = 0; i < C->L; i++) {
        uint64_t ncell = (uint64_t)1 << (d * C->I[i]);
        int64_t* o = calloc(ncell + 1, sizeof(int64_t));
        for (int64_t p = C->lstart[i]; p < C->lstart[i + 1]; p++) o[rec[p].cell + 1]++;
        for (uint64_t cidx = 0; cidx < ncell; cidx++) o[cidx + 1] += o[cidx];
        C->offs[i] = o;
    }
    free(rec);
    free(lay);
    return 0;
}

static void cp_free(cp_ctx* C) {
    free(C->t2);
    free(C->order);
    for (int i = 0; i < MAXL; i++) free(C->offs[i]);
    free(C->E);
    free(C->sh);
}

/* Tables exported for tests: L, lcap, Dmax, then I[L], CL[L][L], counts[L],
 * wmax[L] (as doubles in wtab). */
static void export_tables(cp_ctx* C, int32_t* itab, double* wtab) {
    if (itab) {
        itab[0] = C->L;
        itab[1] = C->lcap;
        itab[2] = C->Dmax;
        for (int i = 0; i < C->L; i++) itab[3 + i] = C->I[i];
        for (int i = 0; i < C->L; i++)
            for (int j = 0; j < C->L; j++) itab[3 + MAXL + i * MAXL + j] = C->CL[i][j];
    }
    if (wtab) {
        for (int i = 0; i < C->L; i++) {
            wtab[i] = C->wmax[i];
            wtab[MAXL + i] = (double)C->lcount[i];
        }
    }
}

/* Oracle 2 for GIRGs.  order_out (n entries, may be NULL) receives the sorted
 * vertex order; stats (8 + 3*33 entries) the counters and, per level, the
 * visited neighbouring, distant and (A, A) cell pairs; items/items_cap an optional
 * item log; skip_sampling enumerates items without drawing. */
int64_t orc_girg_cellpairs(int64_t n, int d, const uint32_t* X, const double* w, double w_min,
                           double W, double T, double K, uint64_t seed, uint32_t* edges,
                           int64_t cap, int64_t* stats, int64_t* order_out, int32_t* itab,
                           double* wtab, int64_t* items, int64_t items_cap, int64_t* n_items,
                           int skip_sampling, int lcap_override) {
    cp_ctx C;
    memset(&C, 0, sizeof(C));
    C.model = 0;
    C.n = n;
    C.d = d;
    C.seed = seed;
    C.X = X;
    C.w = w;
    girg_model_init(&C.M, d, T, K, W);
    C.edges = edges;
    C.cap = cap;
    C.items = items;
    C.items_cap = items_cap;
    C.skip_sampling = skip_sampling;
    cp_prepare(&C, w_min, lcap_override);
    if (n > 0) recur(&C, 0, 0, 0);
    sample_streams(&C);
    if (stats) {
        memcpy(stats, C.stats, sizeof(C.stats));
        memcpy(stats + 8, C.lvl_nb, sizeof(C.lvl_nb));
        memcpy(stats + 8 + 33, C.lvl_far, sizeof(C.lvl_far));
        memcpy(stats + 8 + 66, C.lvl_self, sizeof(C.lvl_self));
    }
    if (order_out) memcpy(order_out, C.order, sizeof(int64_t) * n);
    if (n_items) *n_items = C.n_items;
    export_tables(&C, itab, wtab);
    int64_t m = C.error ? -1 : C.m;
    cp_free(&C);
    return m;
}

/* Oracle 2 for HRGs through the mapping of Sec. 2.3 (d = 1, weights
 * e^((R-r)/2) with unit 1). */
int64_t orc_hrg_cellpairs(int64_t n, const uint32_t* X, const double* r, double R, double T,
                          uint64_t seed, uint32_t* edges, int64_t cap, int64_t* stats,
                          int64_t* order_out, int32_t* itab, double* wtab, int64_t* items,
                          int64_t items_cap, int64_t* n_items, int skip_sampling,
                          int lcap_override) {
    cp_ctx C;
    memset(&C, 0, sizeof(C));
    C.model = 1;
    C.n = n;
    C.d = 1;
    C.seed = seed;
    C.X = X;
    C.r = r;
    hrg_model_init(&C.H, T, R);
    double* w = malloc(sizeof(double) * (n ? n : 1));
    C.E = malloc(sizeof(double) * (n ? n : 1));
    C.sh = malloc(sizeof(double) * (n ? n : 1));
    for (int64_t v = 0; v < n; v++) {
        w[v] = orc_hrg_weight(r[v], R);
        C.E[v] = orc_det_exp(r[v]);
        C.sh[v] = (C.E[v] - 1.0 / C.E[v]) * 0.5;
    }
    C.w = w;
    C.edges = edges;
    C.cap = cap;
    C.items = items;
    C.items_cap = items_cap;
    C.skip_sampling = skip_sampling;
    cp_prepare(&C, 1.0, lcap_override);
    if (n > 0) recur(&C, 0, 0, 0);
    sample_streams(&C);
    if (stats) {
        memcpy(stats, C.stats, sizeof(C.stats));
        memcpy(stats + 8, C.lvl_nb, sizeof(C.lvl_nb));
        memcpy(stats + 8 + 33, C.lvl_far, sizeof(C.lvl_far));
        memcpy(stats + 8 + 66, C.lvl_self, sizeof(C.lvl_self));
    }
    if (order_out) memcpy(order_out, C.order, sizeof(int64_t) * n);
    if (n_items) *n_items = C.n_items;
    export_tables(&C, itab, wtab);
    int64_t m = C.error ? -1 : C.m;
    cp_free(&C);
    free(w);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Expected average degree and the search for the scale (Sec. 4.1, App. B.2) */
/* ------------------------------------------------------------------------ */

static int cmp_desc(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return x > y ? -1 : (x < y ? 1 : 0);
}

/* For a pair u != v let z = 2^d K w_u w_v / W.  Integrating Eq. 1 over the
 * uniform position of v on the torus (an L-infinity ball of volume (2r)^d):
 * p = 1 for r^d <= K q, so if z >= 1 the whole torus (r <= 1/2) gives p = 1 and
 * E[X_uv] = 1 (the pairs E_R of App. B.2); otherwise
 *   E[X_uv] = z / (1 - T) - T z^(1/T) / (1 - T)   (T > 0),   z   (T = 0).
 * f(K) = (1/n) sum over ordered pairs u != v.  With the weights sorted in
 * decreasing order, the E_R partners of u are a prefix (w_v >= 1 / (A w_u),
 * A = 2^d K / W) and the other partners the suffix; their sums of w_v and of
 * w_v^(1/T) come from suffix sums accumulated from the light end, the latter as
 * a log-sum-exp so that no power of a weight is ever formed (z^(1/T) < 1 on the
 * suffix, while w^(1/T) alone leaves the range of doubles for small T). */
typedef struct {
    int64_t n;
    int d;
    double T, W;
    double* ws;  /* weights, decreasing */
    double* lw;  /* their logarithms */
    double* suf; /* suf[i] = sum_{j >= i} ws[j] */
    double* lse; /* lse[i] = log sum_{j >= i} exp(lw[j] / T) (T > 0) */
} deg_ctx;

static void deg_init(deg_ctx* G, int64_t n, int d, double T, const double* w, double W) {
    G->n = n;
    G->d = d;
    G->T = T;
    G->W = W;
    size_t sz = sizeof(double) * (size_t)(n + 1);
    G->ws = malloc(sz);
    G->lw = malloc(sz);
    G->suf = malloc(sz);
    G->lse = malloc(sz);
    memcpy(G->ws, w, sizeof(double) * (size_t)n);
    qsort(G->ws, (size_t)n, sizeof(double), cmp_desc);
    G->suf[n] = 0.0;
    G->lse[n] = -INFINITY;
    for (int64_t i = n - 1; i >= 0; i--) {
        G->lw[i] = log(G->ws[i]);
        G->suf[i] = G->suf[i + 1] + G->ws[i];
        if (T > 0.0) {
            double b = G->lw[i] / T; /* the largest term of the suffix from i */
            G->lse[i] = b + log1p(exp(G->lse[i + 1] - b));
        }
    }
}

static void deg_free(deg_ctx* G) {
    free(G->ws);
    free(G->lw);
    free(G->suf);
    free(G->lse);
}

static double deg_f(const deg_ctx* G, double K) {
    const int64_t n = G->n;
    const double T = G->T, A = ldexp(K, G->d) / G->W, lA = log(A);
    double total = 0.0;
    int64_t k = n; /* E_R partners of u: indices < k (shrinks as w_u decreases) */
    for (int64_t u = 0; u < n; u++) {
        while (k > 0 && A * G->ws[u] * G->ws[k - 1] < 1.0) k--;
        double cnt = (double)k - (u < k ? 1.0 : 0.0);
        /* suffix [k, n) without u */
        double sw, ls;
        if (u < k) {
            sw = G->suf[k];
            ls = G->lse[k];
        } else if (u == k) {
            sw = G->suf[k + 1];
            ls = G->lse[k + 1];
        } else {
            sw = G->suf[k] - G->ws[u];
            ls = T > 0.0 ? G->lse[k] + log1p(-exp(G->lw[u] / T - G->lse[k])) : 0.0;
        }
        double z_sum = A * G->ws[u] * sw;
        double e = z_sum;
        if (T > 0.0) {
            double zt_sum = exp((lA + G->lw[u]) / T + ls); /* sum of z^(1/T) */
            e = (z_sum - T * zt_sum) / (1.0 - T);
        }
        total += cnt + e;
    }
    return total / (double)n;
}

double orc_girg_avg_degree(double K, int64_t n, int d, double T, const double* w, double W) {
    deg_ctx G;
    deg_init(&G, n, d, T, w, W);
    double f = deg_f(&G, K);
    deg_free(&G);
    return f;
}

/* The scale K with f(K) = target: f increases with K.  Start from the K at
 * which the E_R-free sum alone reaches the target, bracket by doubling or
 * halving, then bisect on log K until the bracket is 1e-13 relative. */
double orc_girg_solve_K(double target, int64_t n, int d, double T, const double* w, double W) {
    deg_ctx G;
    deg_init(&G, n, d, T, w, W);
    double s2 = 0.0;
    for (int64_t i = n - 1; i >= 0; i--) s2 += G.ws[i] * G.ws[i];
    double K0 = target * (double)n * W * (T > 0.0 ? 1.0 - T : 1.0) / (ldexp(1.0, d) * (W * W - s2));
    if (!(K0 > 1e-300 && K0 < 1e300)) K0 = 1.0;
    double lo = K0, hi = K0;
    if (deg_f(&G, K0) < target) {
        while (deg_f(&G, hi) < target && hi < 1e300) hi *= 2.0;
        lo = hi / 2.0;
    } else {
        while (deg_f(&G, lo) >= target && lo > 1e-300) lo /= 2.0;
        hi = lo * 2.0;
    }
    for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; it++) {
        double mid = sqrt(lo * hi);
        if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
        if (deg_f(&G, mid) < target)
            lo = mid;
        else
            hi = mid;
    }
    deg_free(&G);
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------ HRG degree
 * The paper states only that R = 2 ln n + C with C setting the average degree
 * (Sec. 2.2); the oracle computes the expected average degree from the model's
 * definition.  Two vertices are independent with radius density
 * alpha sinh(alpha r) / (cosh(alpha R) - 1) on [0, R] and uniform angles, so
 * E[deg] = (n - 1) P(edge).  With G(t) = P(dist < t) for two random vertices:
 *   T = 0:  P(edge) = G(R)  (edge iff dist < R);
 *   T > 0:  P(edge) = E[p_T(dist)] = E[G(t)] for t logistic with location R and
 *           scale 2T, since p_T(x) = 1/(exp((x - R)/2T) + 1) is the probability
 *           that such a t exceeds x.
 * G(t) = int int f(r1) f(r2) Phi(r1, r2, t) dr1 dr2, where Phi is the fraction of
 * angle differences in [0, pi] with dist < t: 1 if t >= r1 + r2, 0 if
 * t <= |r1 - r2|, else (2/pi) asin(sqrt((cosh t - cosh(r1 - r2)) /
 * (2 sinh r1 sinh r2))) by the law of cosines of Sec. 2.2.
 *
 * Quadrature: in y = R - r; every interval between the points where Phi stops
 * being smooth is mapped by y = a + (b - a)(1 - cos s)/2, s in [0, pi] (which
 * absorbs the square-root behaviour of Phi at those points) and integrated by
 * composite Gauss-Legendre rules; the region where Phi = 1 uses the radial CDF
 * in closed form.  The t integral uses the same rule on panels growing
 * geometrically away from R, truncated where the logistic weight is below
 * e^-40. */

#define HRG_GL_M 8     /* Gauss-Legendre points per panel */
#define HRG_Y_PANELS 4 /* panels per smooth interval in y */
#define HRG_T_PANELS 2 /* panels per t interval */

static double hrg_glx[HRG_GL_M], hrg_glw[HRG_GL_M];
static int hrg_gl_ready = 0;

/* Nodes and weights of the m-point Gauss-Legendre rule on [-1, 1], by Newton's
 * method on the Legendre polynomial P_m (three-term recurrence). */
static void gauss_legendre(int m, double* x, double* w) {
    for (int i = 0; i < m; i++) {
        double z = cos(M_PI * (i + 0.75) / (m + 0.5)), pm = 0.0, dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            pm = p1;
            dp = m * (z * p1 - p0) / (z * z - 1.0);
            double dz = pm / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

typedef struct {
    double alpha, R, chR; /* chR = cosh(alpha R) - 1 */
} hrg_radial;

/* density and CDF of y = R - r */
static double hrg_fy(const hrg_radial* H, double y) {
    return H->alpha * sinh(H->alpha * (H->R - y)) / H->chR;
}
static double hrg_Fy(const hrg_radial* H, double y) {
    return (H->chR - (cosh(H->alpha * (H->R - y)) - 1.0)) / H->chR;
}

static double hrg_phi(double r1, double r2, double t, double cht) {
    if (t >= r1 + r2) return 1.0;
    if (t <= fabs(r1 - r2)) return 0.0;
    double s = (cht - cosh(r1 - r2)) / (2.0 * sinh(r1) * sinh(r2));
    if (s <= 0.0) return 0.0;
    if (s >= 1.0) return 1.0;
    return (2.0 / M_PI) * asin(sqrt(s));
}

/* int_a^b g(y) dy with y = a + (b - a)(1 - cos s)/2 and `panels` Gauss-Legendre
 * panels on s in [0, pi]: fills nodes and weights, returns their number. */
static int cos_rule(double a, double b, int panels, double* y, double* wt) {
    int k = 0;
    for (int p = 0; p < panels; p++) {
        double s0 = M_PI * p / panels, s1 = M_PI * (p + 1) / panels;
        for (int i = 0; i < HRG_GL_M; i++) {
            double s = 0.5 * (s0 + s1) + 0.5 * (s1 - s0) * hrg_glx[i];
            y[k] = a + (b - a) * (1.0 - cos(s)) * 0.5;
            wt[k] = 0.5 * (s1 - s0) * hrg_glw[i] * (b - a) * 0.5 * sin(s);
            k++;
        }
    }
    return k;
}

/* G(t) = P(dist < t) for two independent random vertices. */
static double hrg_dist_cdf(const hrg_radial* H, double t) {
    const double R = H->R;
    if (t <= 0.0) return 0.0;
    if (t >= 2.0 * R) return 1.0;
    const double cht = cosh(t);
    double bp[5];
    int nb = 0;
    bp[nb++] = 0.0;
    double cand[3] = {R - t, 2.0 * R - t, t};
    for (int q = 0; q < 3; q++)
        if (cand[q] > 0.0 && cand[q] < R) bp[nb++] = cand[q];
    bp[nb++] = R;
    for (int a = 1; a < nb; a++) /* sort the few breakpoints */
        for (int b = a; b > 0 && bp[b] < bp[b - 1]; b--) {
            double tmp = bp[b];
            bp[b] = bp[b - 1];
            bp[b - 1] = tmp;
        }
    double y1s[HRG_Y_PANELS * HRG_GL_M], w1s[HRG_Y_PANELS * HRG_GL_M];
    double y2s[HRG_Y_PANELS * HRG_GL_M], w2s[HRG_Y_PANELS * HRG_GL_M];
    double total = 0.0;
    for (int iv = 0; iv + 1 < nb; iv++) {
        if (!(bp[iv + 1] > bp[iv])) continue;
        int k1 = cos_rule(bp[iv], bp[iv + 1], HRG_Y_PANELS, y1s, w1s);
        for (int a = 0; a < k1; a++) {
            double y1 = y1s[a], r1 = R - y1;
            double c1 = y1 - t > 0.0 ? y1 - t : 0.0; /* Phi > 0 only for y2 in (c1, c2) */
            double c2 = y1 + t < R ? y1 + t : R;
            double b1 = 2.0 * R - t - y1; /* Phi = 1 for y2 >= b1 */
            if (!(c2 > c1)) continue;
            double inner = 0.0;
            if (b1 <= c1) {
                inner = hrg_Fy(H, c2) - hrg_Fy(H, c1);
            } else {
                double hi = c2 < b1 ? c2 : b1;
                int k2 = cos_rule(c1, hi, HRG_Y_PANELS, y2s, w2s);
                for (int b = 0; b < k2; b++)
                    inner += w2s[b] * hrg_fy(H, y2s[b]) * hrg_phi(r1, R - y2s[b], t, cht);
                if (b1 < c2) inner += hrg_Fy(H, c2) - hrg_Fy(H, b1);
            }
            total += w1s[a] * hrg_fy(H, y1) * inner;
        }
    }
    return total;
}

/* Probability of an edge between two random vertices. */
static double hrg_edge_prob(double alpha, double T, double R) {
    if (!hrg_gl_ready) {
        gauss_legendre(HRG_GL_M, hrg_glx, hrg_glw);
        hrg_gl_ready = 1;
    }
    hrg_radial H = {alpha, R, cosh(alpha * R) - 1.0};
    if (T == 0.0) return hrg_dist_cdf(&H, R);
    /* logistic density of t: e / (2T (1 + e)^2), e = exp(-|t - R| / 2T) */
    const double s = 2.0 * T, lo = R - 40.0 * s > 0.0 ? R - 40.0 * s : 0.0;
    const double hi = R + 40.0 * s < 2.0 * R ? R + 40.0 * s : 2.0 * R;
    double edges_t[2 * 64 + 2];
    int ne = 0;
    double ws = s;
    double x = R;
    double left[64];
    int nl = 0;
    while (x > lo && nl < 64) {
        x = x - ws > lo ? x - ws : lo;
        left[nl++] = x;
        ws *= 2.0;
    }
    for (int q = nl - 1; q >= 0; q--) edges_t[ne++] = left[q];
    edges_t[ne++] = R;
    x = R;
    ws = s;
    while (x < hi && ne < 2 * 64 + 1) {
        x = x + ws < hi ? x + ws : hi;
        edges_t[ne++] = x;
        ws *= 2.0;
    }
    double ts[HRG_T_PANELS * HRG_GL_M], wts[HRG_T_PANELS * HRG_GL_M];
    double total = 0.0;
    for (int q = 0; q + 1 < ne; q++) {
        if (!(edges_t[q + 1] > edges_t[q])) continue;
        int k = cos_rule(edges_t[q], edges_t[q + 1], HRG_T_PANELS, ts, wts);
        for (int a = 0; a < k; a++) {
            double e = exp(-fabs(ts[a] - R) / s);
            double dens = e / (s * (1.0 + e) * (1.0 + e));
            total += wts[a] * dens * hrg_dist_cdf(&H, ts[a]);
        }
    }
    /* t above the truncation: G = 1 there when hi = 2R, and the logistic mass
     * beyond R + 40 s is below e^-40 otherwise */
    double eh = exp(-(hi - R) / s);
    total += eh / (1.0 + eh);
    return total;
}

double orc_hrg_avg_degree(int64_t n, double alpha, double T, double R) {
    return (double)(n - 1) * hrg_edge_prob(alpha, T, R);
}

/* The R with expected average degree `target`: E[deg] decreases in R; bracket by
 * unit steps from 2 ln n, then bisect to a relative width of 1e-12. */
double orc_hrg_solve_R(int64_t n, double alpha, double T, double target) {
    double lo = 2.0 * log((double)n), hi = lo;
    if (orc_hrg_avg_degree(n, alpha, T, lo) >= target) {
        hi = lo + 1.0;
        while (orc_hrg_avg_degree(n, alpha, T, hi) >= target && hi < 600.0) {
            lo = hi;
            hi += 1.0;
        }
    } else {
        lo = hi - 1.0;
        while (lo > 1e-3 && orc_hrg_avg_degree(n, alpha, T, lo) < target) {
            hi = lo;
            lo = lo - 1.0 > 1e-3 ? lo - 1.0 : 1e-3;
        }
    }
    for (int it = 0; it < 200 && hi - lo > 1e-12 * hi; it++) {
        double mid = 0.5 * (lo + hi);
        if (orc_hrg_avg_degree(n, alpha, T, mid) >= target)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Threshold model (T = 0), brute force: for each vertex u of us[0..nu), every v != u
 * with r^d <= K w_u w_v / W, written as (u, v) pairs (u < v not required); returns
 * the number of pairs (at most cap are written).  For checking sampled vertices of
 * graphs too large for the samplers above. */
int64_t orc_girg_thresh_neighbors(int64_t n, int d, const uint32_t* X, const double* w, double W,
                                  double K, const int64_t* us, int64_t nu, int64_t* out,
                                  int64_t cap) {
    girg_model M;
    girg_model_init(&M, d, 0.0, K, W);
    int64_t m = 0;
    for (int64_t a = 0; a < nu; a++) {
        int64_t u = us[a];
        for (int64_t v = 0; v < n; v++) {
            if (v == u) continue;
            uint32_t D = torus_dist(X + u * d, X + v * d, d);
            if (girg_thresh_edge(&M, w[u], w[v], D)) {
                if (m < cap) {
                    out[2 * m] = u;
                    out[2 * m + 1] = v;
                }
                m++;
            }
        }
    }
    return m;
}
