// Vertex generation and weight reductions (Sec. 2.1, Sec. 2.2, Sec. 5.1 steps 1-3).
//
// Weights are Pareto by inversion, w = w_min U^(-1/(beta-1)), positions are
// 32-bit fixed-point torus coordinates, HRG radii invert the CDF
// (cosh(alpha r) - 1) / (cosh(alpha R) - 1); every draw is a Philox4x32-10
// counter keyed by the seed.  The reduction pass sums the weights exactly in
// 128-bit fixed point (so W is the exactly rounded sum), counts the buckets and
// takes their largest weights (and HRG radius ranges), and optionally the FP64
// sums the degree formula of App. B.2 needs.
#include "internal.cuh"
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

// Reductions over the weights (and radii for HRG) of all vertices.
__global__ void k_reduce(int64_t n, const double* __restrict__ w, const double* __restrict__ r,
                         double w_min, int E0, int want_sums, double invT, int m_int,
                         Reduce* __restrict__ out) {
    __shared__ unsigned int s_cnt[kMaxLayers];
    __shared__ unsigned long long s_wmax[kMaxLayers];
    __shared__ unsigned long long s_rmin[kMaxLayers];
    __shared__ unsigned long long s_rmax[kMaxLayers];
    __shared__ unsigned long long s_lo[32], s_hi[32];
    __shared__ double s_sum[3][32];
    for (int t = threadIdx.x; t < kMaxLayers; t += blockDim.x) {
        s_cnt[t] = 0;
        s_wmax[t] = 0;
        s_rmin[t] = ~0ull;
        s_rmax[t] = 0;
    }
    __syncthreads();
    unsigned long long lo = 0, hi = 0;
    double a2 = 0.0, at = 0.0, a2t = 0.0;
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
        const int layer = layer_of(wv, w_min);
        atomicAdd(&s_cnt[layer], 1u);
        atomicMax(&s_wmax[layer], b);
        if (r) {
            const unsigned long long rb = double_to_bits(r[v]);
            atomicMin(&s_rmin[layer], rb);
            atomicMax(&s_rmax[layer], rb);
        }
        if (want_sums) {
            a2 += wv * wv;
            if (invT > 0.0) {
                // w^(1/T) by repeated products when 1/T is a small integer
                double t;
                if (m_int > 0) {
                    t = wv;
                    for (int q = 1; q < m_int; ++q) t *= wv;
                } else {
                    t = exp2(invT * log2(wv));
                }
                at += t;
                a2t += t * t;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long tlo = __shfl_down_sync(0xffffffffu, lo, o);
        const unsigned long long thi = __shfl_down_sync(0xffffffffu, hi, o);
        add128(lo, hi, tlo, thi);
        a2 += __shfl_down_sync(0xffffffffu, a2, o);
        at += __shfl_down_sync(0xffffffffu, at, o);
        a2t += __shfl_down_sync(0xffffffffu, a2t, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (range_err) atomicOr(&out->range_error, 1u);
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
        s_sum[0][warp] = a2;
        s_sum[1][warp] = at;
        s_sum[2][warp] = a2t;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        lo = lane < nw ? s_lo[lane] : 0ull;
        hi = lane < nw ? s_hi[lane] : 0ull;
        a2 = lane < nw ? s_sum[0][lane] : 0.0;
        at = lane < nw ? s_sum[1][lane] : 0.0;
        a2t = lane < nw ? s_sum[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long tlo = __shfl_down_sync(0xffffffffu, lo, o);
            const unsigned long long thi = __shfl_down_sync(0xffffffffu, hi, o);
            add128(lo, hi, tlo, thi);
            a2 += __shfl_down_sync(0xffffffffu, a2, o);
            at += __shfl_down_sync(0xffffffffu, at, o);
            a2t += __shfl_down_sync(0xffffffffu, a2t, o);
        }
        if (lane == 0) {
            const unsigned long long old = atomicAdd(&out->sum_lo, lo);
            const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
            atomicAdd(&out->sum_hi, hi + carry);
            if (want_sums) {
                atomicAdd(&out->s2, a2);
                atomicAdd(&out->st, at);
                atomicAdd(&out->s2t, a2t);
            }
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
}

// Weights above a threshold, for the error term of App. B.2.
__global__ void k_gather_above(int64_t n, const double* __restrict__ w, double thr,
                               double* __restrict__ out, unsigned int cap,
                               unsigned int* __restrict__ count) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const double wv = w[v];
        if (wv > thr) {
            const unsigned int s = atomicAdd(count, 1u);
            if (s < cap) out[s] = wv;
        }
    }
}

// Weight threshold for the heaviest weights the search for c will need (App. B.2):
// 0.9 times the weight below which no vertex has a partner in E_R at the c0 where
// the leading term of f(c) reaches the target.  The root lies at or a little above
// c0, where that weight is smaller; the search starts at c0 and fetches more weights
// only if it moves further.  One thread; an estimate, so CUDA's pow is good enough.
__global__ void k_top_threshold(const Reduce* __restrict__ red, int64_t n, int d, double T,
                                double target, int E0, double* __restrict__ thr) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double W = ldexp((double)red->sum_hi * 0x1p64 + (double)red->sum_lo, E0);
    double wmax = 0.0;
    for (int i = 0; i < 64; ++i)
        if (red->cnt[i]) wmax = fmax(wmax, __longlong_as_double((long long)red->wmax[i]));
    const double S1 = W - red->s2 / W, two_d = ldexp(1.0, d);
    double qs;
    if (T > 0.0) {
        const double c0 = pow(target * (double)n * (1.0 - T) / (two_d * S1), 1.0 / T);
        qs = 1.0 / (two_d * pow(c0, T));
    } else {
        const double c0 = pow(target * (double)n / (two_d * S1), 1.0 / d);
        qs = 1.0 / (two_d * pow(c0, (double)d));
    }
    const double t = 0.9 * qs * W / wmax;
    *thr = (t > 0.0 && t < 1e300) ? t : 0.0;
}

__global__ void k_gather_above_dev(int64_t n, const double* __restrict__ w,
                                   const double* __restrict__ thr, double* __restrict__ out,
                                   unsigned int cap, unsigned int* __restrict__ count) {
    const double t = *thr;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const double wv = w[v];
        if (wv > t) {
            const unsigned int s = atomicAdd(count, 1u);
            if (s < cap) out[s] = wv;
        }
    }
}

// Sort the gathered weights in decreasing order (one block, bitonic network in
// shared memory on the bit patterns, which order positive doubles); count[1] = 1
// when sorted, 0 when there were more than kTopSortMax.
__global__ void __launch_bounds__(1024) k_sort_top(double* __restrict__ buf,
                                                   unsigned int* __restrict__ count) {
    extern __shared__ unsigned long long s_key[];
    const unsigned int k = count[0];
    if (k > kTopSortMax) {
        if (threadIdx.x == 0) count[1] = 0u;
        return;
    }
    unsigned int m = 1;
    while (m < k) m <<= 1;
    for (unsigned int i = threadIdx.x; i < m; i += blockDim.x)
        s_key[i] = i < k ? (unsigned long long)__double_as_longlong(buf[i]) : 0ull;
    __syncthreads();
    for (unsigned int size = 2; size <= m; size <<= 1) {
        for (unsigned int stride = size >> 1; stride > 0; stride >>= 1) {
            for (unsigned int i = threadIdx.x; i < m; i += blockDim.x) {
                const unsigned int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;  // final order: decreasing
                    const unsigned long long a = s_key[i], b = s_key[j];
                    if (desc ? (a < b) : (a > b)) {
                        s_key[i] = b;
                        s_key[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (unsigned int i = threadIdx.x; i < k; i += blockDim.x)
        buf[i] = __longlong_as_double((long long)s_key[i]);
    if (threadIdx.x == 0) count[1] = 1u;
}

// ------------------------------------------------------------------ launchers
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
    k_girg_points<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(n, d, expo, w_min, (uint32_t)seed,
                                                             (uint32_t)(seed >> 32), w, X);
}

void launch_hrg_points(int64_t n, double alpha, double R, uint64_t seed, double* r, double* w,
                       uint32_t* X, cudaStream_t st) {
    const double ea = det_exp(alpha * R);
    const double cosh_aR = (ea + 1.0 / ea) * 0.5;
    ++g_launches;
    k_hrg_points<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(n, alpha, cosh_aR - 1.0, R,
                                                            (uint32_t)seed, (uint32_t)(seed >> 32),
                                                            r, w, X);
}

void launch_min_weight(int64_t n, const double* w, unsigned long long* out, cudaStream_t st) {
    ++g_launches;
    k_min_weight<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, w, out);
}

void launch_reduce(int64_t n, const double* w, const double* r, double w_min, int E0,
                   int want_sums, double invT, Reduce* out, cudaStream_t st) {
    ++g_launches;
    int m_int = 0;
    if (invT > 0.0 && invT == floor(invT) && invT <= 64.0) m_int = (int)invT;
    k_reduce<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, w, r, w_min, E0, want_sums, invT,
                                                        m_int, out);
}

void launch_gather_above(int64_t n, const double* w, double thr, double* out, unsigned int cap,
                         unsigned int* count, cudaStream_t st) {
    ++g_launches;
    k_gather_above<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, w, thr, out, cap, count);
}

void launch_top_weights(int64_t n, const double* w, const Reduce* red, int d, double T,
                        double target, int E0, double* thr, double* out, unsigned int cap,
                        unsigned int* count, cudaStream_t st) {
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_sort_top, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(kTopSortMax * sizeof(unsigned long long))) ==
               cudaSuccess;
    }();
    (void)attr;
    g_launches += 3;
    k_top_threshold<<<1, 32, 0, st>>>(red, n, d, T, target, E0, thr);
    k_gather_above_dev<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, w, thr, out, cap, count);
    k_sort_top<<<1, 1024, kTopSortMax * sizeof(unsigned long long), st>>>(out, count);
}

}  // namespace gg
