// The geometric data structure of Sec. 3.4 / Lemma 1: every vertex gets the key
// (bucket, Morton code of its cell at the bucket's insertion level) as one dense
// global cell index; a histogram over the cells plus an exclusive scan gives
// the prefix sums P_C of all buckets at once.  The vertex order (ties by original
// id) then comes from placing each vertex by those prefix sums and ranking it among
// the ids of its cell, or, where cells hold many vertices on average, from a stable
// LSD radix sort of (key, id) as in Sec. 4.4 (bucket first, Morton code second).
// The gather kernels lay out the sorted per-vertex arrays (structure of arrays,
// coalesced).
#include "internal.cuh"
#include "kernels.h"
#include "layers.cuh"

namespace gg {

struct KeyTab {
    int8_t I[kMaxLayers];
    uint32_t base[kMaxLayers + 1];
};

__global__ void k_keys(int64_t n, int d, const double* __restrict__ w, const uint32_t* __restrict__ X,
                       double w_min, KeyTab tab, uint32_t* __restrict__ key,
                       uint32_t* __restrict__ val, uint32_t* __restrict__ cnt, bool slots) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int layer = layer_of_bits(w[v], w_min);
        const int lev = tab.I[layer];
        uint32_t coord[kMaxDim];
        for (int k = 0; k < d; ++k) coord[k] = lev ? (X[(int64_t)k * n + v] >> (32 - lev)) : 0u;
        const uint32_t code = lev ? morton_encode(coord, d) : 0u;
        const uint32_t kk = tab.base[layer] + code;
        key[v] = kk;
        // slots: the arrival slot of v in its cell (placement by counts); else v (radix sort)
        const uint32_t slot = atomicAdd(&cnt[kk], 1u);
        val[v] = slots ? slot : (uint32_t)v;
    }
}

// ------------------------------------------------------------------ scan
// Exclusive scans: 32-bit counts into 32- or 64-bit prefixes (reduce per tile,
// scan of the tile sums, down-sweep).
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T block_exclusive_scan(T x, T* s_warp, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        T v = lane < nw ? s_warp[lane] : T(0);
        T vi = v;
        for (int o = 1; o < 32; o <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += t;
        }
        if (lane < nw) s_warp[lane] = vi - v;
        if (lane == 31) s_warp[32] = vi;
    }
    __syncthreads();
    const T r = s_warp[warp] + incl - x;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

// n_dev (optional): the length is min(*n_dev, n), read on the device.
__device__ __forceinline__ int64_t scan_len(int64_t n, const unsigned long long* n_dev) {
    if (!n_dev) return n;
    const unsigned long long m = *n_dev;
    return m < (unsigned long long)n ? (int64_t)m : n;
}

template <class Tin, class T>
__global__ void k_scan_reduce(const Tin* __restrict__ in, int64_t n, T* __restrict__ sums,
                              const unsigned long long* __restrict__ n_dev) {
    __shared__ T s_warp[33];
    n = scan_len(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= n) {  // past the end: an empty tile
        if (threadIdx.x == 0) sums[blockIdx.x] = T(0);
        return;
    }
    T acc = 0;
    for (int it = 0; it < kScanItems; ++it) {
        const int64_t i = base + (int64_t)it * kScanThreads + threadIdx.x;
        if (i < n) acc += (T)in[i];
    }
    T total;
    block_exclusive_scan<T>(acc, s_warp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Tile staging in shared memory: one pad element per 128 bytes, so that both the
// striped (coalesced global) and the blocked (16 consecutive items per thread) accesses
// are free of bank conflicts for 4- and 8-byte elements.
template <class E>
__device__ __forceinline__ int stage_pos(int i) {
    return i + (i >> (sizeof(E) == 8 ? 4 : 5));
}
constexpr int kStageWords = (kScanTile + kScanTile / 16) * 2;  // 8-byte elements, padded

template <class Tin, class T>
__global__ void k_scan_down(const Tin* in, T* out, int64_t n, const T* __restrict__ prefix,
                            const unsigned long long* __restrict__ n_dev) {
    static_assert(sizeof(Tin) == 4 || sizeof(Tin) == 8, "4- or 8-byte inputs");
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte prefixes");
    __shared__ __align__(16) uint32_t s_buf[kStageWords];
    __shared__ T s_warp[33];
    n = scan_len(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= n) return;  // uniform per block
    const int tid = threadIdx.x;
    const int64_t rem = n - base;
    const int m = rem < kScanTile ? (int)rem : kScanTile;  // items of this tile
    // the tile, striped (coalesced), into shared memory; zeros past the end
    Tin* s_in = reinterpret_cast<Tin*>(s_buf);
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        const int i = it * kScanThreads + tid;
        s_in[stage_pos<Tin>(i)] = i < m ? in[base + i] : Tin(0);
    }
    __syncthreads();
    T v[kScanItems];
    T acc = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        v[it] = (T)s_in[stage_pos<Tin>(tid * kScanItems + it)];
        acc += v[it];
    }
    T total;  // block_exclusive_scan ends with a barrier: s_in is free after it
    T run = block_exclusive_scan<T>(acc, s_warp, &total) + (prefix ? prefix[blockIdx.x] : T(0));
    T* s_out = reinterpret_cast<T*>(s_buf);
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        s_out[stage_pos<T>(tid * kScanItems + it)] = run;
        run += v[it];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        const int i = it * kScanThreads + tid;
        if (i < m) out[base + i] = s_out[stage_pos<T>(i)];
    }
}

size_t scan_tmp_words(int64_t n) {
    size_t words = 0;
    int64_t m = n;
    while (m > kScanTile) {
        m = (m + kScanTile - 1) / kScanTile;
        words += (size_t)m + 32;
    }
    return words + 64;
}

// n: the length, or with n_dev its upper bound (the grid is sized for n; tiles past
// *n_dev are empty).
template <class Tin, class T>
static void scan_impl(const Tin* in, T* out, int64_t n, T* tmp, cudaStream_t st,
                      const unsigned long long* n_dev = nullptr) {
    if (n <= 0) return;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        ++g_launches;
        k_scan_down<Tin, T><<<1, kScanThreads, 0, st>>>(in, out, n, nullptr, n_dev);
        return;
    }
    T* sums = tmp;
    ++g_launches;
    k_scan_reduce<Tin, T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums, n_dev);
    scan_impl<T, T>(sums, sums, nb, tmp + nb + 32, st);
    ++g_launches;
    k_scan_down<Tin, T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums, n_dev);
}

void launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t st) {
    scan_impl<uint32_t, uint32_t>(in, out, n, tmp, st);
}

void launch_scan_u32_to_u64(const uint32_t* in, unsigned long long* out, int64_t n,
                            unsigned long long* tmp, cudaStream_t st) {
    scan_impl<uint32_t, unsigned long long>(in, out, n, tmp, st);
}

void launch_scan_u32_to_u64_dev(const uint32_t* in, unsigned long long* out,
                                const unsigned long long* n_dev, int64_t n_max,
                                unsigned long long* tmp, cudaStream_t st) {
    scan_impl<uint32_t, unsigned long long>(in, out, n_max, tmp, st, n_dev);
}

// ------------------------------------------------------------------ radix sort
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // 2048 = 8 warps x 8 rounds x 32

__global__ void k_radix_hist(const uint32_t* __restrict__ key, int64_t n, int shift,
                             uint32_t* __restrict__ hist, uint32_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
        const int64_t i = base + (int64_t)it * kRadixThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint32_t* __restrict__ key, const uint32_t* __restrict__ val, int64_t n,
                int shift, const uint32_t* __restrict__ hist, uint32_t ntiles,
                uint32_t* __restrict__ key_out, uint32_t* __restrict__ val_out) {
    __shared__ uint32_t wcnt[8][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < 8 * 256; t += kRadixThreads) (&wcnt[0][0])[t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile + warp * 256;
    uint32_t k[kRadixItems], v[kRadixItems], rank[kRadixItems];
    int dig[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        k[r] = valid ? key[i] : 0u;
        v[r] = valid ? val[i] : 0u;
        const int dg = (int)((k[r] >> shift) & 255u);
        dig[r] = valid ? dg : -1;
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const bool bit = (dg >> b) & 1;
            const uint32_t bm = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bm : ~bm;
        }
        uint32_t before = 0;
        if (valid) before = wcnt[warp][dg];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][dg] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    {
        uint32_t run = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        if (dig[r] >= 0) {
            const uint32_t pos =
                hist[(size_t)dig[r] * ntiles + blockIdx.x] + wcnt[warp][dig[r]] + rank[r];
            key_out[pos] = k[r];
            val_out[pos] = v[r];
        }
    }
}

size_t radix_tmp_words(int64_t n) {
    const int64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
    return (size_t)(256 * ntiles) + scan_tmp_words(256 * ntiles) + 64;
}

void radix_sort_pairs(uint32_t* key, uint32_t* val, uint32_t* key_alt, uint32_t* val_alt,
                      int64_t n, int bits, uint32_t* tmp, cudaStream_t st, uint32_t** key_out,
                      uint32_t** val_out) {
    const uint32_t ntiles = (uint32_t)((n + kRadixTile - 1) / kRadixTile);
    uint32_t* hist = tmp;
    uint32_t* stmp = tmp + (size_t)256 * ntiles + 32;
    uint32_t *ki = key, *vi = val, *ko = key_alt, *vo = val_alt;
    for (int shift = 0; shift < bits; shift += 8) {
        ++g_launches;
        k_radix_hist<<<ntiles, kRadixThreads, 0, st>>>(ki, n, shift, hist, ntiles);
        launch_scan_u32(hist, hist, (int64_t)256 * ntiles, stmp, st);
        ++g_launches;
        k_radix_scatter<<<ntiles, kRadixThreads, 0, st>>>(ki, vi, n, shift, hist, ntiles, ko, vo);
        uint32_t* t = ki;
        ki = ko;
        ko = t;
        t = vi;
        vi = vo;
        vo = t;
    }
    *key_out = ki;
    *val_out = vi;
}

static int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b > max_blocks) b = max_blocks;
    if (b < 1) b = 1;
    return (int)b;
}

// ------------------------------------------------------------------ doubles, decreasing
// Positive doubles order like their bit patterns, so the complemented patterns in
// increasing order are the values in decreasing order: two stable radix sorts, by the
// low word and then by the high word, order the 64-bit patterns.
__global__ void k_f64_words(const double* __restrict__ x, int64_t n, uint32_t* __restrict__ lo,
                            uint32_t* __restrict__ hi, uint32_t* __restrict__ idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = ~(unsigned long long)__double_as_longlong(x[i]);
        lo[i] = (uint32_t)b;
        hi[i] = (uint32_t)(b >> 32);
        idx[i] = (uint32_t)i;
    }
}

__global__ void k_gather_words(const uint32_t* __restrict__ src, const uint32_t* __restrict__ perm,
                               int64_t n, uint32_t* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

__global__ void k_gather_doubles(const double* __restrict__ src, const uint32_t* __restrict__ perm,
                                 int64_t n, double* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

size_t sort_desc_words(int64_t n) { return (size_t)5 * (size_t)n + radix_tmp_words(n) + 64; }

void sort_f64_desc(const double* in, int64_t n, double* out, uint32_t* words, cudaStream_t st) {
    if (n <= 0) return;
    uint32_t* lo = words;
    uint32_t* hi = lo + n;
    uint32_t* idx = hi + n;
    uint32_t* ka = idx + n;
    uint32_t* va = ka + n;
    uint32_t* tmp = va + n;
    const int grid = grid_for(n, 256, device_sms() * 16);
    ++g_launches;
    k_f64_words<<<grid, 256, 0, st>>>(in, n, lo, hi, idx);
    uint32_t *k1, *p1;
    radix_sort_pairs(lo, idx, ka, va, n, 32, tmp, st, &k1, &p1);  // by the low word
    uint32_t* kfree = k1 == lo ? ka : lo;
    uint32_t* vfree = p1 == idx ? va : idx;
    ++g_launches;
    k_gather_words<<<grid, 256, 0, st>>>(hi, p1, n, kfree);  // high words in that order
    uint32_t *k2, *p2;
    radix_sort_pairs(kfree, p1, k1, vfree, n, 32, tmp, st, &k2, &p2);  // then by the high word
    ++g_launches;
    k_gather_doubles<<<grid, 256, 0, st>>>(in, p2, n, out);
}

// ------------------------------------------------------------------ placement by counts
// The same order without the radix passes.  With the cell histogram scanned (offs[c] =
// first sorted position of cell c, offs[C] = n), a vertex goes to offs[key] plus its
// arrival slot in the cell (key and id as one 8-byte record: the placement is a random
// scatter, and one write per vertex touches half the sectors of two).  Arrival order is
// not deterministic, so k_rank then puts
// each vertex at offs[key] + (the number of smaller ids in its cell): the order of the
// stable sort (ties by original id).  Cells with more than kRankMax vertices are copied
// as they are and sorted afterwards, one block per cell (k_sort_cells).
constexpr uint32_t kRankMax = 64;

__global__ void k_place(int64_t n, const uint32_t* __restrict__ key,
                        const uint32_t* __restrict__ slot, const uint32_t* __restrict__ offs,
                        uint2* __restrict__ kt) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = key[v];
        kt[offs[c] + slot[v]] = make_uint2(c, (uint32_t)v);  // one scattered 8-byte write
    }
}

__global__ void k_rank(int64_t n, const uint2* __restrict__ kt, const uint32_t* __restrict__ offs,
                       uint32_t* __restrict__ skey, uint32_t* __restrict__ sid,
                       uint32_t* __restrict__ big, uint32_t* __restrict__ nbig, uint32_t big_cap) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint2 e = kt[p];
        const uint32_t c = e.x, v = e.y;
        const uint32_t a = offs[c], b = offs[c + 1];
        skey[p] = c;
        if (b - a > kRankMax) {  // a large cell: copied, sorted by k_sort_cells
            sid[p] = v;
            if ((uint32_t)p == a) {
                const uint32_t q = atomicAdd(nbig, 1u);
                if (q < big_cap) big[q] = c;
            }
            continue;
        }
        uint32_t r = 0;
        for (uint32_t q = a; q < b; ++q) r += kt[q].y < v ? 1u : 0u;
        sid[a + r] = v;
    }
}

// One block per large cell: a bitonic network over the cell's ids in place, on the
// cell padded to a power of two P with +inf (a comparator whose upper element lies past
// the end never swaps, so those comparators are skipped).  Each merge starts with the
// mirrored comparator (i, i ^ (size - 1)), so every comparator puts the smaller id
// first.  The ids stay in global memory; the barrier after each stage orders them
// within the block.
__global__ void __launch_bounds__(256) k_sort_cells(const uint32_t* __restrict__ offs,
                                                    const uint32_t* __restrict__ big,
                                                    const uint32_t* __restrict__ nbig,
                                                    uint32_t big_cap, uint32_t* sid) {
    uint32_t nb = *nbig;
    if (nb > big_cap) nb = big_cap;
    for (uint32_t q = blockIdx.x; q < nb; q += gridDim.x) {
        const uint32_t c = big[q];
        uint32_t* x = sid + offs[c];
        const uint32_t m = offs[c + 1] - offs[c];
        uint64_t P = 1;
        while (P < m) P <<= 1;
        const uint32_t half = (uint32_t)(P >> 1);
        for (int lg = 1; (1ull << lg) <= P; ++lg) {
            const uint32_t size = 1u << lg;
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                const bool mirror = stride == (size >> 1);
                for (uint32_t t = threadIdx.x; t < half; t += blockDim.x) {
                    const uint32_t i = (t / stride) * 2u * stride + (t % stride);
                    const uint32_t j = mirror ? (i ^ (size - 1u)) : i + stride;
                    if (j < m) {
                        const uint32_t lo = x[i], hi = x[j];
                        if (lo > hi) {
                            x[i] = hi;
                            x[j] = lo;
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
}

size_t place_tmp_words(int64_t n) { return (size_t)(n / (kRankMax + 1)) + 2; }

void place_by_counts(const uint32_t* key, const uint32_t* slot, const uint32_t* offs, int64_t n,
                     uint2* kt, uint32_t* skey, uint32_t* sid, uint32_t* tmp, cudaStream_t st) {
    const uint32_t big_cap = (uint32_t)(place_tmp_words(n) - 1);
    uint32_t* nbig = tmp;  // zeroed by the caller
    uint32_t* big = tmp + 1;
    const int grid = grid_for(n, 256, device_sms() * 16);
    g_launches += 3;
    k_place<<<grid, 256, 0, st>>>(n, key, slot, offs, kt);
    k_rank<<<grid, 256, 0, st>>>(n, kt, offs, skey, sid, big, nbig, big_cap);
    k_sort_cells<<<device_sms() * 2, 256, 0, st>>>(offs, big, nbig, big_cap, sid);
}

// ------------------------------------------------------------------ gathers
// Per-vertex scale s with kappa_uv = s_u s_v (kappa: distance at which p = 1, or the
// threshold distance at T = 0): log2 s = (log2 w - log2(W)/2) / d + gamma.  Only the
// single-precision fast path uses it; its error is covered by the decision band.
// The sorted GIRG vertex arrays: weights and buckets, and either packed records (rec,
// d <= 4: coordinates, scale and id of a vertex in 16 or 32 bytes, so that a pair test
// reads each vertex with one or two vector loads) or the separate coordinate and scale
// arrays (Xs, sv).
__global__ void k_gather_girg(int64_t n, int d, const uint32_t* __restrict__ perm,
                              const uint32_t* __restrict__ X, const double* __restrict__ w,
                              double w_min, double log2W_half, float gamma, float invd,
                              uint32_t* __restrict__ Xs, double* __restrict__ ws,
                              float* __restrict__ sv, uint8_t* __restrict__ slayer,
                              uint4* __restrict__ rec) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = perm[p];
        const double wv = w[v];
        ws[p] = wv;
        const float s = exp2f((log2f((float)wv) - (float)log2W_half) * invd + gamma);
        slayer[p] = (uint8_t)layer_of_bits(wv, w_min);
        if (rec) {
            uint32_t x[4] = {0u, 0u, 0u, 0u};
            for (int k = 0; k < d && k < 4; ++k) x[k] = X[(int64_t)k * n + v];
            if (d <= 2) {
                rec[p] = make_uint4(x[0], x[1], __float_as_uint(s), v);
            } else {
                rec[2 * p] = make_uint4(x[0], x[1], x[2], x[3]);
                rec[2 * p + 1] = make_uint4(__float_as_uint(s), v, 0u, 0u);
            }
        } else {
            for (int k = 0; k < d; ++k) Xs[(int64_t)k * n + p] = X[(int64_t)k * n + v];
            sv[p] = s;
        }
    }
}

__global__ void k_scale(int64_t n, const double* __restrict__ w, double log2W_half, float gamma,
                        float invd, float* __restrict__ sv) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        sv[p] = exp2f((log2f((float)w[p]) - (float)log2W_half) * invd + gamma);
}

__global__ void k_gather_hrg(int64_t n, const uint32_t* __restrict__ perm,
                             const uint32_t* __restrict__ X, const double* __restrict__ r,
                             const double* __restrict__ w, uint32_t* __restrict__ Xs,
                             double* __restrict__ rs, float* __restrict__ E32,
                             float* __restrict__ einv32, float* __restrict__ sh32,
                             uint8_t* __restrict__ slayer, uint4* __restrict__ hrec) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = perm[p];
        Xs[p] = X[v];
        const double rv = r[v];
        rs[p] = rv;
        const float rf = (float)rv;
        const float E = expf(rf), ei = expf(-rf), sh = sinhf(rf);
        if (hrec) {
            hrec[p] = make_uint4(X[v], __float_as_uint(E), __float_as_uint(ei), __float_as_uint(sh));
        } else {
            E32[p] = E;
            einv32[p] = ei;
            sh32[p] = sh;
        }
        slayer[p] = (uint8_t)layer_of_bits(w[v], 1.0);
    }
}

void launch_keys(int64_t n, int d, const double* w, const uint32_t* X, double w_min,
                 const int8_t* I, const uint32_t* layer_base, uint32_t* key, uint32_t* val,
                 uint32_t* cnt, bool slots, cudaStream_t st) {
    KeyTab tab;
    memcpy(tab.I, I, sizeof(tab.I));
    memcpy(tab.base, layer_base, sizeof(tab.base));
    ++g_launches;
    k_keys<<<grid_for(n, 256, device_sms() * 16), 256, 0, st>>>(n, d, w, X, w_min, tab, key, val, cnt, slots);
}

void launch_gather_girg(int64_t n, int d, const uint32_t* perm, const uint32_t* X,
                        const double* w, double w_min, double log2W_half, float gamma,
                        float invd, uint32_t* Xs, double* ws, float* sv, uint8_t* slayer,
                        uint4* rec, cudaStream_t st) {
    ++g_launches;
    k_gather_girg<<<grid_for(n, 256, device_sms() * 16), 256, 0, st>>>(
        n, d, perm, X, w, w_min, log2W_half, gamma, invd, Xs, ws, sv, slayer, rec);
}

void launch_scale(int64_t n, const double* w, double log2W_half, float gamma, float invd,
                  float* sv, cudaStream_t st) {
    ++g_launches;
    k_scale<<<grid_for(n, 256, device_sms() * 16), 256, 0, st>>>(n, w, log2W_half, gamma, invd, sv);
}

void launch_gather_hrg(int64_t n, const uint32_t* perm, const uint32_t* X, const double* r,
                       const double* w, uint32_t* Xs, double* rs, float* E32, float* einv32,
                       float* sh32, uint8_t* slayer, uint4* hrec, cudaStream_t st) {
    ++g_launches;
    k_gather_hrg<<<grid_for(n, 256, device_sms() * 16), 256, 0, st>>>(n, perm, X, r, w, Xs, rs, E32,
                                                             einv32, sh32, slayer, hrec);
}

}  // namespace gg
