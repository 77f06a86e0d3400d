// Vertex generation and weight reductions (Sec. 2.1, Sec. 2.2, Sec. 5.1 steps 1-3).
//
// Weights are Pareto by inversion, w = w_min U^(-1/(beta-1)), positions are
// 32-bit fixed-point torus coordinates, HRG radii invert the CDF
// (cosh(alpha r) - 1) / (cosh(alpha R) - 1); every draw is a Philox4x32-10
// counter keyed by the seed.  The reduction pass sums the weights exactly in
// 128-bit fixed point (so W is the exactly rounded sum), counts the buckets and
// takes their largest weights (and HRG radius ranges), and optionally the FP64
// sums the degree formula of App. B.2 needs.
#include <atomic>
#include "internal.cuh"
#include "layers.cuh"
#include "kernels.h"

namespace gg {

__global__ void k_girg_points(int64_t n, int d, double expo, double w_min, uint32_t s0,
                              uint32_t s1, double* __restrict__ w, uint32_t* __restrict__ X) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t vlo = (uint32_t)v, vhi = (uint32_t)((uint64_t)v >> 32);
        const P4 o = philox(vlo, vhi, kTagWeight, 0u, s0, s1);
        const double U = uniform53(o.x, o.y);
        w[v] = DMUL(w_min, det_pow(U, expo));
        for (int k = 0; k < d; k += 4) {
            const P4 q = philox(vlo, vhi, kTagPos, (uint32_t)(k >> 2), s0, s1);
            X[(int64_t)k * n + v] = q.x;
            if (k + 1 < d) X[(int64_t)(k + 1) * n + v] = q.y;
            if (k + 2 < d) X[(int64_t)(k + 2) * n + v] = q.z;
            if (k + 3 < d) X[(int64_t)(k + 3) * n + v] = q.w;
        }
    }
}

__global__ void k_hrg_points(int64_t n, double alpha, double cosh_aR_m1, double R, uint32_t s0,
                             uint32_t s1, double* __restrict__ r, double* __restrict__ w,
                             uint32_t* __restrict__ X) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t vlo = (uint32_t)v, vhi = (uint32_t)((uint64_t)v >> 32);
        const P4 o = philox(vlo, vhi, kTagRadius, 0u, s0, s1);
        const double U = uniform53(o.x, o.y);
        const double rv = DDIV(det_acosh(DADD(1.0, DMUL(U, cosh_aR_m1))), alpha);
        const P4 q = philox(vlo, vhi, kTagPos, 0u, s0, s1);
        X[v] = q.x;
        if (r) r[v] = rv;
        if (w) w[v] = det_exp(DMUL(DSUB(R, rv), 0.5));  // HRG -> GIRG weight (Sec. 2.3)
    }
}

// Smallest weight (bit pattern of a positive double orders like the value).
__global__ void k_min_weight(int64_t n, const double* __restrict__ w,
                             unsigned long long* __restrict__ out) {
    unsigned long long m = ~0ull;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = double_to_bits(w[v]);
        m = b < m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_down_sync(0xffffffffu, m, o);
        m = t < m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(out, m);
}

__device__ __forceinline__ void add128(unsigned long long& lo, unsigned long long& hi,
                                       unsigned long long blo, unsigned long long bhi) {
    const unsigned long long s = lo + blo;
    hi += bhi + (s < lo ? 1ull : 0ull);
    lo = s;
}

__device__ __forceinline__ bool last_block(unsigned int* ticket);
__device__ void top_threshold(Reduce* __restrict__ red, const double* __restrict__ part_s2,
                              int nb, int64_t n, int d, double T, double target, int E0,
                              double* __restrict__ thr);

// Reductions over the weights (and radii for HRG) of all vertices.
__global__ void k_reduce(int64_t n, const double* __restrict__ w, const double* __restrict__ r,
                         double w_min, int E0, double* __restrict__ part_s2,
                         Reduce* __restrict__ out, ThresholdJob job) {
    __shared__ unsigned int s_cnt[kMaxLayers];
    __shared__ unsigned long long s_wmax[kMaxLayers];
    __shared__ unsigned long long s_rmin[kMaxLayers];
    __shared__ unsigned long long s_rmax[kMaxLayers];
    __shared__ unsigned long long s_lo[32], s_hi[32];
    __shared__ double s_sum[32];
    for (int t = threadIdx.x; t < kMaxLayers; t += blockDim.x) {
        s_cnt[t] = 0;
        s_wmax[t] = 0;
        s_rmin[t] = ~0ull;
        s_rmax[t] = 0;
    }
    __syncthreads();
    unsigned long long lo = 0, hi = 0;
    double a2 = 0.0;
    int range_err = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const double wv = w[v];
        const unsigned long long b = double_to_bits(wv);
        const int eb = (int)((b >> 52) & 0x7ff);
        const unsigned long long mant = (b & 0x000fffffffffffffull) | (1ull << 52);
        // w = mant 2^(eb - 1075) = (mant << sh) 2^E0; terms < 2^96 keep 2^31 of them
        // inside 128 bits
        const int sh = eb - 1075 - E0;
        if (sh < 0 || sh > 43) {
            range_err = 1;
        } else if (sh == 0) {
            add128(lo, hi, mant, 0ull);
        } else {
            add128(lo, hi, mant << sh, mant >> (64 - sh));
        }
        const int layer = layer_of_bits(wv, w_min);
        // most weights share the lowest layers: one count increment per layer and
        // warp, and the extremes only when they improve on the block's (a stale read
        // costs one more atomic, never a wrong result)
        const unsigned int peers = __match_any_sync(__activemask(), layer);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&s_cnt[layer], (unsigned)__popc(peers));
        if (b > s_wmax[layer]) atomicMax(&s_wmax[layer], b);
        if (r) {
            const unsigned long long rb = double_to_bits(r[v]);
            if (rb < s_rmin[layer]) atomicMin(&s_rmin[layer], rb);
            if (rb > s_rmax[layer]) atomicMax(&s_rmax[layer], rb);
        }
        if (part_s2) a2 += wv * wv;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long tlo = __shfl_down_sync(0xffffffffu, lo, o);
        const unsigned long long thi = __shfl_down_sync(0xffffffffu, hi, o);
        add128(lo, hi, tlo, thi);
        a2 += __shfl_down_sync(0xffffffffu, a2, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (range_err) atomicOr(&out->range_error, 1u);
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
        s_sum[warp] = a2;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        lo = lane < nw ? s_lo[lane] : 0ull;
        hi = lane < nw ? s_hi[lane] : 0ull;
        a2 = lane < nw ? s_sum[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long tlo = __shfl_down_sync(0xffffffffu, lo, o);
            const unsigned long long thi = __shfl_down_sync(0xffffffffu, hi, o);
            add128(lo, hi, tlo, thi);
            a2 += __shfl_down_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            const unsigned long long old = atomicAdd(&out->sum_lo, lo);
            const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
            atomicAdd(&out->sum_hi, hi + carry);
            if (part_s2) part_s2[blockIdx.x] = a2;  // summed in block order later
        }
    }
    for (int t = threadIdx.x; t < kMaxLayers; t += blockDim.x) {
        if (s_cnt[t]) {
            atomicAdd(&out->cnt[t], (unsigned long long)s_cnt[t]);
            atomicMax(&out->wmax[t], s_wmax[t]);
            if (r) {
                atomicMin(&out->rmin[t], s_rmin[t]);
                atomicMax(&out->rmax[t], s_rmax[t]);
            }
        }
    }
    // the split threshold, by the last block once every block's sums are in
    if (job.thr && last_block(&out->blocks_done))
        top_threshold(out, part_s2, gridDim.x, n, job.d, job.T, job.target, E0, job.thr);
}


// Fixed-order sum of a per-block partial array by one block of 256 threads
// (deterministic; loads through L2, as the last block of a grid reads the partials
// the other blocks wrote).
__device__ double block_ordered_sum(const double* __restrict__ part, int nb) {
    __shared__ double s[256];
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += __ldcg(part + i);
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

// True in the last block of the grid to get here (after __threadfence, so that the
// writes of every other block are visible to it).  *ticket starts at 0.
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    return s_last;
}

// The split threshold of the degree model (App. B.2): the weight above which a
// vertex can have partners in E_R at the scale K0 where the sum of
// 2^d K w_u w_v / (W (1 - T)) over all pairs reaches the target, divided by a
// margin.  The root K lies at or above K0 (the capping of E_R pairs and the
// z^(1/T) terms only lower f), where that weight is smaller: K / K0 stays below
// about 1.3 for T < 0.7 and 2.3 up to T = 0.9 (beta >= 2.1, degree <= 32), hence
// margins 1.4 and 2.8; the search fetches a new split only if it moves further.
// One block (256 threads): also finishes sum w^2 in block order.
__device__ void top_threshold(Reduce* __restrict__ red, const double* __restrict__ part_s2,
                              int nb, int64_t n, int d, double T, double target, int E0,
                              double* __restrict__ thr) {
    __shared__ unsigned long long s_wmax;  // bits of the largest weight (positive doubles
                                           // order like their bit patterns)
    if (threadIdx.x == 0) s_wmax = 0ull;
    const double s2 = block_ordered_sum(part_s2, nb);  // synchronises the block
    if (threadIdx.x < 64 && __ldcg(&red->cnt[threadIdx.x]))
        atomicMax(&s_wmax, __ldcg(&red->wmax[threadIdx.x]));
    __syncthreads();
    if (threadIdx.x != 0) return;
    red->s2 = s2;
    const double W = ldexp((double)__ldcg(&red->sum_hi) * 0x1p64 + (double)__ldcg(&red->sum_lo), E0);
    const double wmax = __longlong_as_double((long long)s_wmax);
    const double K0 = target * (double)n * W * (T > 0.0 ? 1.0 - T : 1.0) /
                      (ldexp(W * W - s2, d));
    const double margin = T >= 0.7 ? 2.8 : 1.4;
    const double t = W / (margin * ldexp(K0, d) * wmax);
    *thr = (t > 0.0 && t < 1e300) ? t : 0.0;
}

// One pass over the weights at the threshold: the weights above it are appended to
// `out` (count[0]), and each block writes its sums over the weights at or below it:
// sum w, sum w^2, sum (w/thr)^(1/T), sum (w/thr)^(2/T) (powers <= 1).
__global__ void k_split_weights(int64_t n, const double* __restrict__ w,
                                const double* __restrict__ thr, double invT, int m_int,
                                double* __restrict__ out, unsigned int cap,
                                unsigned int* __restrict__ count, double* __restrict__ part,
                                double* __restrict__ sums) {
    __shared__ double s[4][8];
    const double t = *thr, inv_t = 1.0 / t;  // only feeds the search for K: no exact rounding needed
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const double wv = w[v];
        if (wv > t) {
            const unsigned int slot = atomicAdd(count, 1u);
            if (slot < cap) out[slot] = wv;
        } else {
            a[0] += wv;
            a[1] += wv * wv;
            if (invT > 0.0) {
                const double x = fmin(wv * inv_t, 1.0);
                double y;
                if (m_int > 0) {
                    y = x;
                    for (int q = 1; q < m_int; ++q) y *= x;
                } else {
                    y = det_pow(x, invT);  // integer pipes: the FP64 units are slow
                }
                a[2] += y;
                a[3] += y * y;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        for (int o = 16; o > 0; o >>= 1) a[q] += __shfl_down_sync(0xffffffffu, a[q], o);
        if (lane == 0) s[q][warp] = a[q];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) acc += s[threadIdx.x][i];
        part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = acc;
    }
    // the four sums in a fixed order, by the last block: 64 threads per sum, each over
    // every 64th partial, then a fixed tree within the group
    if (last_block(&count[2])) {
        static_assert(sizeof(s) >= 8 * sizeof(double), "group results fit the block buffer");
        const int nb = gridDim.x, q = threadIdx.x >> 6, g = threadIdx.x & 63;
        double a = 0.0;
        for (int i = g; i < nb; i += 64) a += __ldcg(part + (size_t)q * nb + i);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        __syncthreads();  // s is reused
        if ((threadIdx.x & 31) == 0) s[0][threadIdx.x >> 5] = a;  // 8 warp results
        __syncthreads();
        if (threadIdx.x < 4) sums[threadIdx.x] = s[0][2 * threadIdx.x] + s[0][2 * threadIdx.x + 1];
    }
}

// The gathered weights in decreasing order, when there are at most kTopSortMax of them
// (count[1] = 1; else count[1] = 0 and the host has them sorted): each weight goes to its
// rank, the number of larger weights plus the number of equal ones before it.  A block
// ranks kRankPerBlock weights with kRankSplit threads each, every thread counting over
// every kRankSplit-th weight of shared memory; k weights cost k^2 comparisons over
// ceil(k / kRankPerBlock) blocks.  They compare the bit patterns as integers (positive
// doubles order like them), since the FP64 units are slow.
constexpr unsigned int kRankThreads = 256;
constexpr unsigned int kRankSplit = 8;
constexpr unsigned int kRankPerBlock = kRankThreads / kRankSplit;

__global__ void __launch_bounds__(kRankThreads) k_rank_top(const double* __restrict__ buf,
                                                          unsigned int* __restrict__ count,
                                                          double* __restrict__ sorted) {
    __shared__ unsigned long long s_w[kTopSortMax];
    const unsigned int k = count[0];
    if (k > kTopSortMax) {
        if (blockIdx.x == 0 && threadIdx.x == 0) count[1] = 0u;
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) count[1] = 1u;
    if (blockIdx.x * kRankPerBlock >= k) return;  // the whole block: no weight of its own
    for (unsigned int i = threadIdx.x; i < k; i += kRankThreads)
        s_w[i] = (unsigned long long)__double_as_longlong(buf[i]);
    __syncthreads();
    const unsigned int i = blockIdx.x * kRankPerBlock + threadIdx.x / kRankSplit;
    const unsigned int sub = threadIdx.x % kRankSplit;
    unsigned int r = 0;
    unsigned long long x = 0;
    if (i < k) {
        x = s_w[i];
        for (unsigned int j = sub; j < k; j += kRankSplit)
            r += (j < i ? s_w[j] >= x : s_w[j] > x) ? 1u : 0u;  // ties before i count
    }
    // the kRankSplit partial counts of a weight sit in consecutive lanes
#pragma unroll
    for (unsigned int o = kRankSplit / 2; o > 0; o >>= 1)
        r += __shfl_down_sync(0xffffffffu, r, o, kRankSplit);
    if (i < k && sub == 0) sorted[r] = __longlong_as_double((long long)x);
}

bool det_tables_gen() { return det_tables_ready(); }

// ------------------------------------------------------------------ launchers
int device_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
            v = 1;
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

static int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b > max_blocks) b = max_blocks;
    if (b < 1) b = 1;
    return (int)b;
}

void launch_girg_points(int64_t n, int d, double beta, double w_min, uint64_t seed, double* w,
                        uint32_t* X, cudaStream_t st) {
    const double expo = -1.0 / (beta - 1.0);
    ++g_launches;
    k_girg_points<<<grid_for(n, 256, device_sms() * 32), 256, 0, st>>>(n, d, expo, w_min, (uint32_t)seed,
                                                             (uint32_t)(seed >> 32), w, X);
}

void launch_hrg_points(int64_t n, double alpha, double R, uint64_t seed, double* r, double* w,
                       uint32_t* X, cudaStream_t st) {
    const double ea = det_exp(alpha * R);
    const double cosh_aR = (ea + 1.0 / ea) * 0.5;
    ++g_launches;
    k_hrg_points<<<grid_for(n, 256, device_sms() * 32), 256, 0, st>>>(n, alpha, cosh_aR - 1.0, R,
                                                            (uint32_t)seed, (uint32_t)(seed >> 32),
                                                            r, w, X);
}

void launch_min_weight(int64_t n, const double* w, unsigned long long* out, cudaStream_t st) {
    ++g_launches;
    k_min_weight<<<grid_for(n, 256, device_sms() * 8), 256, 0, st>>>(n, w, out);
}

// At least eight weights a thread: each block ends in FP64 shuffle trees (four of them in
// the split), which cost as much as the weights themselves on the slow FP64 pipes when a
// thread holds only a few; at most 1216 blocks, enough loads in flight at large n.
int reduce_blocks(int64_t n) { return grid_for((n + 7) / 8, 256, 1216); }

void launch_reduce(int64_t n, const double* w, const double* r, double w_min, int E0,
                   double* part_s2, Reduce* out, cudaStream_t st, const ThresholdJob* job) {
    ++g_launches;
    ThresholdJob j{};
    if (job && part_s2) j = *job;
    k_reduce<<<reduce_blocks(n), 256, 0, st>>>(n, w, r, w_min, E0, part_s2, out, j);
}



// ---------------------------------------------------------------- HRG degree
// The distance CDF of the HRG's expected degree at T > 0 (Sec. 2.2): the probability
// that two random vertices lie closer than t.  Radii have density
// alpha sinh(alpha r) / (cosh(alpha R) - 1); in y = R - r the share of angle
// differences with distance below t is (2/pi) asin(sqrt(s)),
// s = (cosh t - cosh(r1 - r2)) / (2 sinh r1 sinh r2), between the ends where it is 0
// or 1, so the integral runs over the intervals between 0, R and the kinks R - t,
// 2R - t and t.  One block per t node; every thread takes (interval, y1 node, y2 node)
// triples of the product rule, and the block sums them in a fixed order.
constexpr int kCdfThreads = 256;

__device__ __forceinline__ double disk_dens(double alpha, double R, double cm1, double y) {
    return alpha * sinh(alpha * (R - y)) / cm1;
}

__device__ __forceinline__ double disk_cdf(double alpha, double R, double cm1, double y) {
    return 1.0 - (cosh(alpha * (R - y)) - 1.0) / cm1;
}

__device__ __forceinline__ double angle_share(double r1, double r2, double t, double cosh_t) {
    if (t >= r1 + r2) return 1.0;
    if (t <= fabs(r1 - r2)) return 0.0;
    const double s = (cosh_t - cosh(r1 - r2)) / (2.0 * sinh(r1) * sinh(r2));
    if (!(s > 0.0)) return 0.0;
    if (s >= 1.0) return 1.0;
    return 0.63661977236758134308 * asin(sqrt(s));  // 2/pi
}

// Block (node i, interval q) writes the part of P(dist < ts[i]) from the q-th interval
// of y1 to g[4 i + q] (0 where the node has fewer intervals); the host adds the four in
// order.  The interval's y1 nodes, their weights times the radial density and their
// y2 ranges are formed once in shared memory; the threads then take the (y1, y2)
// products.
__global__ void __launch_bounds__(kCdfThreads)
    k_hrg_dist_cdf(double alpha, double R, double cm1, HrgYRule Y,
                   const double* __restrict__ ts, double* __restrict__ g) {
    __shared__ double s_cut[5];
    __shared__ int s_ncut;
    __shared__ double s_f[kHrgYMax], s_y1[kHrgYMax], s_lo[kHrgYMax], s_top[kHrgYMax],
        s_tail[kHrgYMax];
    __shared__ double s_part[kCdfThreads / 32];
    const int q = blockIdx.y;
    double* const out = g + 4 * (size_t)blockIdx.x + q;
    const double t = ts[blockIdx.x];
    if (!(t > 0.0) || t >= 2.0 * R) {
        if (threadIdx.x == 0) *out = (q == 0 && t >= 2.0 * R) ? 1.0 : 0.0;
        return;
    }
    if (threadIdx.x == 0) {
        double c[5];
        int m = 0;
        c[m++] = 0.0;
        c[m++] = R;
        const double cand[3] = {R - t, 2.0 * R - t, t};
        for (int k = 0; k < 3; ++k)
            if (cand[k] > 0.0 && cand[k] < R) c[m++] = cand[k];
        for (int i = 1; i < m; ++i) {  // insertion sort of at most five cuts
            const double x = c[i];
            int j = i - 1;
            while (j >= 0 && c[j] > x) {
                c[j + 1] = c[j];
                --j;
            }
            c[j + 1] = x;
        }
        for (int i = 0; i < m; ++i) s_cut[i] = c[i];
        s_ncut = m;
    }
    __syncthreads();
    const int ny = Y.n;
    if (q >= s_ncut - 1 || !(s_cut[q + 1] > s_cut[q])) {  // no such interval (block-uniform)
        if (threadIdx.x == 0) *out = 0.0;
        return;
    }
    const double a0 = s_cut[q], a1 = s_cut[q + 1];
    if ((int)threadIdx.x < ny) {  // per y1 node: weight times density, y2 range, closed-form tail
        const int a = threadIdx.x;
        const double y1 = a0 + (a1 - a0) * Y.c[a];
        const double lo = fmax(0.0, y1 - t), hi = fmin(R, y1 + t);
        const double full = 2.0 * R - t - y1;  // share = 1 for y2 >= full
        double f = 0.0, tail = 0.0, top = lo;
        if (hi > lo) {
            f = (a1 - a0) * Y.w[a] * disk_dens(alpha, R, cm1, y1);
            if (full <= lo) {
                tail = disk_cdf(alpha, R, cm1, hi) - disk_cdf(alpha, R, cm1, lo);
            } else {
                top = fmin(hi, full);
                if (full < hi) tail = disk_cdf(alpha, R, cm1, hi) - disk_cdf(alpha, R, cm1, full);
            }
        }
        s_f[a] = f;
        s_y1[a] = y1;
        s_lo[a] = lo;
        s_top[a] = top;
        s_tail[a] = tail;
    }
    __syncthreads();
    const double ct = cosh(t);
    double acc = 0.0;
    for (int k = threadIdx.x; k < ny * ny; k += kCdfThreads) {
        const int a = k / ny, b = k % ny;
        const double f = s_f[a];
        if (f == 0.0) continue;
        double in = b == 0 ? s_tail[a] : 0.0;
        const double lo = s_lo[a], top = s_top[a];
        if (top > lo) {
            const double y2 = lo + (top - lo) * Y.c[b];
            in += (top - lo) * Y.w[b] * disk_dens(alpha, R, cm1, y2) *
                  angle_share(R - s_y1[a], R - y2, t, ct);
        }
        acc += f * in;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int i = 0; i < kCdfThreads / 32; ++i) sum += s_part[i];
        *out = sum;
    }
}

void launch_hrg_dist_cdf(double alpha, double R, const HrgYRule& Y, const double* d_ts, int nt,
                         double* d_g, cudaStream_t st) {
    if (nt <= 0) return;
    const double cm1 = cosh(alpha * R) - 1.0;
    ++g_launches;
    k_hrg_dist_cdf<<<dim3(nt, 4), kCdfThreads, 0, st>>>(alpha, R, cm1, Y, d_ts, d_g);
}

void launch_split_weights(int64_t n, const double* w, const double* thr, double T, double* out,
                          unsigned int cap, unsigned int* count, double* part, double* sums,
                          double* sorted, cudaStream_t st) {
    const double invT = T > 0.0 ? 1.0 / T : 0.0;
    int m_int = 0;
    if (invT > 0.0 && invT == floor(invT) && invT <= 64.0) m_int = (int)invT;
    const int nb = reduce_blocks(n);
    g_launches += 2;
    k_split_weights<<<nb, 256, 0, st>>>(n, w, thr, invT, m_int, out, cap, count, part, sums);
    k_rank_top<<<kTopSortMax / kRankPerBlock, kRankThreads, 0, st>>>(out, count, sorted);
}

}  // namespace gg
