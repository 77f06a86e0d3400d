// Device-side configuration, tables and helpers shared by the kernels.
#pragma once
#include <cooperative_groups.h>
#include "common.cuh"

namespace gg {

// Bound p-bar of a type-II item class (bucket pair, level, gap g in {1, 2}), its
// ln(1 - p-bar) and single-precision companions (Sec. 3.2).
struct TwoEntry {
    double pbar;
    double Lb;        // ln(1 - pbar) (0 when pbar = 1)
    float log2pbar;   // log2(pbar) rounded to float
    float invLb;      // 1 / Lb rounded to float (-inf when pbar = 1)
    int32_t k;        // chunk length exponent
    int32_t one;      // pbar == 1 (no jumps: every index is a candidate)
};

// The buckets a row (bucket i, level l, cell A) pairs with: the n2 buckets j >= i
// with CL(i,j) >= l >= 2 (distant cells, type II) at jlist[jbase .. jbase + n2),
// then the n1 buckets with CL(i,j) = l (neighbour cells, type I).  A row has
// n2 6^d + n1 3^d offset combinations, type II first.
struct RowClass {
    uint16_t n2, n1;
    uint32_t jbase;
};

// A type-I item: rectangle V_i^A x V_j^B of sorted positions; bit 31 of b_len
// marks the (A, A, i, i) items that only test pairs at positions a < b.
struct T1Item {
    uint32_t a_begin, a_len, b_begin, b_len;
};

// A type-II stream: geometric jumps over V_i^A x (V_j^B1 ++ V_j^B2 ++ ...), the
// distant partner cells B of A with one gap g, in increasing rank; the partner
// sets are seg_cnt entries of the segment pool from seg_off.
struct alignas(16) Stream {
    uint32_t A;
    uint32_t pack;  // l | i << 5 | j << 11 | (g - 1) << 17 | kTagJump << 18
    uint32_t a_begin, a_len;
    uint32_t seg_off, seg_cnt;
    uint32_t S;     // total size of the partner sets
    uint32_t tii;   // index of its TwoEntry
    uint32_t s0;    // single-chunk streams: offset of the first candidate (draw 0),
                    // already drawn by the enumeration; 0xffffffff otherwise
    float invLb, log2pbar;  // copies of its TwoEntry's fast-path fields
    uint32_t kone;          // its TwoEntry's k | one << 8
};
static_assert(sizeof(Stream) == 48, "stream record layout");
// Work beyond the enumeration is balanced through exclusive prefixes: of the
// pairs of the type-I items and of the chunks of the type-II streams.  A warp
// takes the next range of pairs (chunks) from a 64-bit counter and finds the
// item (stream) of its first pair (chunk) by a search in the prefix.

// One partner set of a stream: its first sorted position and the number of
// positions of the stream's earlier partner sets.
struct Seg {
    uint32_t b_begin, pre;
};


enum : int { kStatT1Pairs = 0, kStatCoins, kStatRecheck, kStatT2Items, kStatDraws,
             kStatCands, kStatRows, kStatT1Items, kStatT2Chunks, kStatEdges,
             kStatLaunches, kStatT1VertexRefs, kStatT1Edges, kStatStreams, kStatChecksum,
             kStatSegs, kStatEnumPasses, kStatEnt2, kStatEnt1, kNumStats };


struct DevCfg {
    int32_t n, d, L, model, precision, tzero, m_int, lcap;
    int32_t n3, n6;  // 3^d and 6^d
    uint32_t seed_lo, seed_hi;
    uint32_t mode;
    double W, K, T, invT, w_min, R, coshR;  // K: scale of Eq. 1 (c^T, or c^d at T = 0)
    float dT;          // d / T (GIRG)
    float bandG;       // band in the log2 domain of decisions
    float band_ratio;  // relative band of kappa / r
    float coshR32;     // cosh R rounded to float (HRG)
    float R32, inv2T32;
    int32_t filt_k;
    int8_t I[kMaxLayers];
    uint8_t CLd[kMaxLayers];
    uint32_t layer_base[kMaxLayers + 1];
    uint32_t lstart[kMaxLayers + 1];
    const TwoEntry* tii;
    const RowClass* classes;  // [i * (kMaxLevel + 1) + l]
    const uint8_t* jlist;
    const uint32_t* offs;
    const uint32_t* Xs;   // d x n sorted coordinates
    const float* sv;      // sorted per-vertex scale (GIRG)
    const double* ws;     // sorted weights (GIRG) / radii (HRG)
    const uint32_t* ids;  // sorted original ids
    const uint32_t* skey; // sorted keys (global cell index at the insertion level)
    const uint8_t* slayer;
    const float* E32;     // HRG e^r, e^-r, sinh r (sorted; null when hrec holds them)
    const float* einv32;
    const float* sh32;
    const uint4* hrec;    // HRG packed records {angle, e^r, e^-r, sinh r} (FP32 bits, sorted)
    // packed sorted GIRG records for d <= 4 (null otherwise; then Xs and sv): d <= 2 one
    // uint4 {x0, x1, scale bits, id} per vertex, d = 3, 4 two {x0, x1, x2, x3},
    // {scale bits, id, 0, 0}
    const uint4* vrec;
    const float* filt_lo;  // HRG distance filter (cosh thresholds), rounded down
    const float* filt_hi;  // rounded up
    void* edges;
    int32_t edge_bytes;
    int64_t cap;
    unsigned long long* edge_count;
    unsigned long long* stats;
    unsigned int* row_count;  // rows found (statistics)
    uint64_t* ent2;           // type-II work entries (row, bucket j)
    unsigned int* ent2_count;
    uint32_t ent2_cap;
    uint64_t* ent1;           // type-I work entries
    unsigned int* ent1_count;
    uint32_t ent1_cap;
    // the entries enumerated in this round: [lo, min(hi, count))
    uint32_t ent2_lo, ent2_hi, ent1_lo, ent1_hi;
    T1Item* t1;
    unsigned long long* t1_count;  // 64-bit: a round may produce more than it holds
    uint32_t t1_cap;
    uint32_t* t1_pairs;                 // pairs per type-I item (a_len * b_len)
    const unsigned long long* t1_pre;   // its exclusive prefix (t1 count + 1 entries)
    Stream* streams;
    unsigned long long* stream_count;
    uint32_t stream_cap;
    uint32_t* stream_chunks;             // chunks per stream (>= 1)
    const unsigned long long* chunk_pre; // its exclusive prefix (stream count + 1 entries)
    Seg* segs;
    unsigned long long* seg_count;
    uint32_t seg_cap;
    unsigned int* error;         // set when a stream needs 2^32 chunks or more
    // optional: 0 when a work list of this round overflowed (its entries past the
    // capacity were not written), and the sampling kernels then do nothing
    const unsigned int* lists_ok;
    uint32_t count_only;         // enumeration: count the work lists, write nothing
    unsigned long long* work64;  // [0] type-I pairs taken, [1] type-II chunks taken
};

// --------------------------------------------------------------- bit tricks
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Put bit b of x at position b * d (x < 2^(32/d)).
__device__ __forceinline__ uint32_t spread_bits(uint32_t x, int d) {
    if (d == 1) return x;
    if (d == 2) {
        x &= 0x0000ffffu;
        x = (x | (x << 8)) & 0x00ff00ffu;
        x = (x | (x << 4)) & 0x0f0f0f0fu;
        x = (x | (x << 2)) & 0x33333333u;
        x = (x | (x << 1)) & 0x55555555u;
        return x;
    }
    if (d == 4) {
        x &= 0xffu;
        x = (x | (x << 12)) & 0x000f000fu;
        x = (x | (x << 6)) & 0x03030303u;
        x = (x | (x << 3)) & 0x11111111u;
        return x;
    }
    uint32_t r = 0;
    for (int b = 0; b * d < 32 && b < 32; ++b) r |= ((x >> b) & 1u) << (b * d);
    return r;
}

// Inverse of spread_bits.
__device__ __forceinline__ uint32_t compact_bits(uint32_t x, int d) {
    if (d == 1) return x;
    if (d == 2) {
        x &= 0x55555555u;
        x = (x | (x >> 1)) & 0x33333333u;
        x = (x | (x >> 2)) & 0x0f0f0f0fu;
        x = (x | (x >> 4)) & 0x00ff00ffu;
        x = (x | (x >> 8)) & 0x0000ffffu;
        return x;
    }
    uint32_t r = 0;
    for (int b = 0; b * d < 32 && b < 32; ++b) r |= ((x >> (b * d)) & 1u) << b;
    return r;
}

// Morton code of cell coordinates at level l (coordinate 0 most significant
// within every d-bit group, Sec. 4.2).
__device__ __forceinline__ uint32_t morton_encode(const uint32_t* coord, int d) {
    uint32_t code = 0;
    for (int k = 0; k < d; ++k) code |= spread_bits(coord[k], d) << (d - 1 - k);
    return code;
}

__device__ __forceinline__ void morton_decode(uint32_t code, int d, uint32_t* coord) {
    for (int k = 0; k < d; ++k) coord[k] = compact_bits(code >> (d - 1 - k), d);
}

// --------------------------------------------------------------- edge output
// Per-warp edge buffer in shared memory, flushed with one global atomic.
constexpr int kEdgeBuf = 256;

struct WarpEdges {
    uint32_t* a;      // kEdgeBuf entries
    uint32_t* b;
    unsigned int* n;  // count (shared)
    unsigned long long mix = 0;  // this lane's share of the checksum of the flushed edges
};

// Order-independent checksum of an edge set: the sum mod 2^64 of the splitmix64
// finalizer (Steele, Lea, Flood, OOPSLA 2014) of u 2^32 + v over the edges (u < v).
__device__ __forceinline__ unsigned long long edge_mix(uint32_t a, uint32_t b) {
    unsigned long long z = ((unsigned long long)a << 32) | b;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void write_edge(const DevCfg& cfg, unsigned long long slot, uint32_t a,
                                           uint32_t b) {
    if (cfg.edge_bytes == 0 || (long long)slot >= cfg.cap) return;  // count-only / overflow
    if (cfg.edge_bytes == 4) {
        reinterpret_cast<uint2*>(cfg.edges)[slot] = make_uint2(a, b);
    } else {
        reinterpret_cast<ulonglong2*>(cfg.edges)[slot] = make_ulonglong2(a, b);
    }
}

// Append one edge (u, v as original ids, any order) from any subset of lanes.
__device__ __forceinline__ void push_edge(const DevCfg& cfg, WarpEdges& we, uint32_t u, uint32_t v) {
    const uint32_t a = u < v ? u : v, b = u < v ? v : u;
    const unsigned int slot = atomicAdd(we.n, 1u);
    if (slot < (unsigned)kEdgeBuf) {
        we.a[slot] = a;
        we.b[slot] = b;
    } else {
        const unsigned long long g = atomicAdd(cfg.edge_count, 1ull);
        write_edge(cfg, g, a, b);
        atomicAdd(&cfg.stats[kStatChecksum], edge_mix(a, b));
    }
}

// Whole warp, once at the end: add the lanes' checksum shares (one atomic per warp).
__device__ __forceinline__ void flush_mix(const DevCfg& cfg, WarpEdges& we) {
    unsigned long long m = we.mix;
    for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&cfg.stats[kStatChecksum], m);
    we.mix = 0;
}

// Whole warp: write out the buffer if it holds at least `threshold` edges.  The
// checksum goes to each lane's share (kLaneMix, for kernels that flush often; added by
// flush_mix at the end) or to one atomic per flush.
template <bool kLaneMix = false>
__device__ __forceinline__ void flush_edges(const DevCfg& cfg, WarpEdges& we, unsigned threshold) {
    __syncwarp();
    unsigned int cnt = *we.n;
    if (cnt > (unsigned)kEdgeBuf) cnt = kEdgeBuf;
    if (cnt >= threshold && cnt > 0) {
        const int lane = threadIdx.x & 31;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cfg.edge_count, (unsigned long long)cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        unsigned long long mix = 0;
        for (unsigned int t = lane; t < cnt; t += 32) {
            write_edge(cfg, base + t, we.a[t], we.b[t]);
            mix += edge_mix(we.a[t], we.b[t]);
        }
        if (kLaneMix) {
            we.mix += mix;
        } else {
            for (int o = 16; o > 0; o >>= 1) mix += __shfl_down_sync(0xffffffffu, mix, o);
            if (lane == 0) atomicAdd(&cfg.stats[kStatChecksum], mix);
        }
        __syncwarp();
        if (lane == 0) *we.n = 0;
    }
    __syncwarp();
}

// --------------------------------------------------------------- uniforms in float
// The uniform U = (2 (bits >> 12) + 1) 2^-53 of two Philox words (bits = hi:lo) in
// single precision, from 32-bit conversions only: U = hi 2^-32 + (2 (lo >> 12) + 1)
// 2^-53 with both terms exact in float and one rounding (relative error <= 2^-23).
__device__ __forceinline__ float uniform32(uint32_t lo, uint32_t hi) {
    return fmaf(__uint2float_rn(2u * (lo >> 12) + 1u), 0x1p-53f, __uint2float_rn(hi) * 0x1p-32f);
}

// 1 - U in single precision: (2^32 - 1 - hi) 2^-32 + (2^21 - 1 - 2 (lo >> 12)) 2^-53.
__device__ __forceinline__ float one_minus_uniform32(uint32_t lo, uint32_t hi) {
    return fmaf(__uint2float_rn(0x1FFFFFu - 2u * (lo >> 12)), 0x1p-53f,
                __uint2float_rn(~hi) * 0x1p-32f);
}

// log2 U from the hardware approximation: U >= 2^-53 is a normal float and
// |log2 U| <= 53, so the absolute error is at most 2 ulp of 64 (2^-17) plus the
// 2^-23 relative rounding of U (2^-22.5): far inside the decision bands.
__device__ __forceinline__ float log2_uniform32(uint32_t lo, uint32_t hi) {
    return __log2f(uniform32(lo, hi));
}

// ln U in single precision with relative error <= 2^-20.5 for all U in (0, 1):
// for U >= 1/2 through ln(1 - (1 - U)); below 1/2 the hardware approximation
// (3 ulp off [1/2, 2], 2^-21.4 absolute at U = 1/2, i.e. 2^-20.9 relative) plus
// the 2^-23 rounding of U.
__device__ __forceinline__ float ln_uniform32(uint32_t lo, uint32_t hi) {
    if (hi >= 0x80000000u) return log1pf(-one_minus_uniform32(lo, hi));
    return __logf(uniform32(lo, hi));
}

// Geometric jump X = floor(ln U / ln(1 - pbar)) against the remaining length rem
// of the chunk.  Returns 0: stop (X >= rem), 1: continue with *X, decided in
// single precision with a 2^-19 relative error bound, or 2: undecided, the
// caller evaluates the FP64 rule.  Only 32-bit conversions (the FP64 units of
// the GPU also convert 64-bit integers).
__device__ __forceinline__ int jump32(uint32_t lo, uint32_t hi, float invLb, unsigned long long rem,
                                      unsigned long long* X) {
    const float x = ln_uniform32(lo, hi) * invLb;  // >= 0
    const float xlo = x * (1.0f - 0x1p-19f), xhi = x * (1.0f + 0x1p-19f);
    if (rem < (1ull << 24)) {
        const float remf = __uint2float_rn((uint32_t)rem);  // exact
        if (xlo >= remf) return 0;
        if (xhi < remf) {
            const float a = floorf(xlo), b = floorf(xhi);
            if (a == b) {
                *X = __float2uint_rz(b);
                return 1;
            }
        }
        return 2;
    }
    const float remf = fmaf(__uint2float_rn((uint32_t)(rem >> 32)), 0x1p32f,
                            __uint2float_rn((uint32_t)rem));
    if (xlo >= remf * (1.0f + 0x1p-20f)) return 0;
    if (xhi < 0x1p22f) {
        const float a = floorf(xlo), b = floorf(xhi);
        if (a == b) {
            *X = __float2uint_rz(b);
            return 1;
        }
    }
    return 2;
}

// The exact FP64 rule: 0 stop, 1 continue with *X.
static __device__ __forceinline__ int jump64(uint32_t lo, uint32_t hi, double Lb, unsigned long long rem,
                                      unsigned long long* X) {
    const double x = floor(DDIV(det_log(uniform53(lo, hi)), Lb));
    if (x >= 0x1p63) return 0;
    const unsigned long long xi = (unsigned long long)x;
    if (xi >= rem) return 0;
    *X = xi;
    return 1;
}

}  // namespace gg
