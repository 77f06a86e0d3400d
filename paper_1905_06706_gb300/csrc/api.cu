// Host orchestration and the C ABI (include/girg_gb300.h).
//
// girg_generate: points -> exact weight sum and bucket statistics -> c (App. B.2)
// -> bucket / level tables (Sec. 3.1) -> keys, prefix sums and radix sort
// (Sec. 3.4, Lemma 1, Sec. 4.4) -> rows -> cell-pair enumeration with inline
// type-II jumps (Algorithm 1, Sec. 3.2) -> type-I tiles -> multi-chunk type-II
// items -> edge count.  The host computes the FP64 tables that every kernel
// reads (comparison and insertion levels, type-II bounds p-bar and ln(1-p-bar)),
// with the same deterministic arithmetic as the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "girg_gb300.h"
#include "internal.cuh"
#include "kernels.h"
#include "layers.cuh"
#include "solver.h"

using namespace gg;

thread_local unsigned long long gg::g_launches = 0;

namespace {

thread_local int64_t g_stats[kNumStats];
thread_local float g_ms[10];

struct CudaFail {
    cudaError_t err;
};
struct Status {
    int code;
};

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) throw CudaFail{e_}; \
    } while (0)

// The library's own memory pool on the current device, created on first use and kept
// until the process exits.  Every call's scratch is taken from it with
// cudaMallocFromPoolAsync and given back with cudaFreeAsync on the call's stream; its
// release threshold is raised so that later calls reuse the freed memory instead of
// returning it to the driver after each synchronisation.  The caller's pools (the
// device's default pool, PyTorch's caching allocator) are left as they are;
// girg_scratch_pool_trim hands the unused part back.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaMemPool_t library_pool() {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxPoolDevices) throw CudaFail{cudaErrorInvalidDevice};
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        CK(cudaMemPoolCreate(&pool, &props));
        uint64_t thr = ~0ull;
        CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

// Scratch allocations from the library's pool, freed on scope exit (stream-ordered),
// unless release() hands them to a longer-lived owner (the resident point-set cache).
// With a reservation, one pool allocation of that size is carved up in order (256-byte
// aligned) and only what does not fit is allocated on its own: a call then makes one or
// two pool calls instead of dozens, on its critical path at the start and at the end.
struct Scratch {
    cudaStream_t st;
    cudaMemPool_t pool;
    std::vector<void*> ptrs;
    size_t bytes = 0;
    char* arena = nullptr;
    size_t arena_cap = 0, arena_used = 0;
    explicit Scratch(cudaStream_t s, size_t reserve = 0) : st(s), pool(library_pool()) {
        if (reserve > 0) {
            void* p = nullptr;
            if (cudaMallocFromPoolAsync(&p, reserve, pool, st) == cudaSuccess) {
                arena = static_cast<char*>(p);
                arena_cap = reserve;
            } else {
                cudaGetLastError();  // no reservation: every request allocates on its own
            }
        }
    }
    template <class T>
    T* get(size_t count) {
        size_t b = count * sizeof(T);
        if (b < 256) b = 256;
        b = (b + 255) & ~(size_t)255;
        bytes += b;
        if (arena && arena_used + b <= arena_cap) {
            T* p = reinterpret_cast<T*>(arena + arena_used);
            arena_used += b;
            return p;
        }
        void* p = nullptr;
        CK(cudaMallocFromPoolAsync(&p, b, pool, st));
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    // the allocations so far, for an owner that outlives this object (no reservation)
    std::vector<void*> release() {
        std::vector<void*> out;
        out.swap(ptrs);
        return out;
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
        if (arena) cudaFreeAsync(arena, st);
    }
};

// Phase marks of one call: CUDA events created once per host thread and device.
struct Timer {
    cudaEvent_t* ev;
    int used = 0;
    cudaStream_t st;
    explicit Timer(cudaStream_t s) : st(s) {
        thread_local cudaEvent_t events[8];
        thread_local int events_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (events_dev != dev) {  // first use on this thread, or another device
            if (events_dev >= 0)
                for (auto& e : events) cudaEventDestroy(e);
            for (auto& e : events) cudaEventCreate(&e);
            events_dev = dev;
        }
        ev = events;
    }
    void mark() {
        if (used < 8) cudaEventRecord(ev[used++], st);
    }
};

double host_ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

double round128(unsigned long long hi, unsigned long long lo, int E0) {
    unsigned __int128 acc = ((unsigned __int128)hi << 64) | lo;
    if (acc == 0) return 0.0;
    int top = 127;
    while (!((acc >> top) & 1)) --top;
    if (top < 53) return std::ldexp((double)(uint64_t)acc, E0);
    const int shift = top - 52;
    unsigned __int128 mant = acc >> shift;
    const unsigned __int128 rem = acc & ((((unsigned __int128)1) << shift) - 1);
    const unsigned __int128 half = ((unsigned __int128)1) << (shift - 1);
    if (rem > half || (rem == half && (mant & 1))) mant += 1;
    return std::ldexp((double)(uint64_t)mant, shift + E0);
}

int bitlen64(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

// Deepest quadtree level by default: floor(32/d) at most (32-bit Morton codes).  At
// T = 0 (type-I items only) deep cells only cut pair tests, down to about 2^(bitlen+4)
// cells.  At T > 0 the type-I pairs of a level (3^d m^2 per cell of m vertices) and its
// distant partner cells (6^d - 3^d per cell) balance near n 2^(-d/2) cells, the level
// floor(log2(n)/d - 1/2) with log2 n = bitlen - 1; timing level caps on GB300 put the
// fastest one there for d = 1..4 and n = 10^6 .. 2^24.
int default_level_cap(int64_t n, int d, double T) {
    int bl = 0;
    while (bl < 63 && ((int64_t)1 << bl) <= n) ++bl;
    int a = 32 / d, b = T > 0.0 ? (2 * bl - 2 - d) / (2 * d) : (bl + 4) / d;
    if (b < 1) b = 1;
    return a < b ? a : b;
}

// Comparison level for the threshold distance kappa: deepest l in [0, cap] with
// 2^-l > kappa (1 + 2^-30) (Sec. 3.1).
int level_for_kappa(double kappa, int cap) {
    const double k2 = kappa * (1.0 + 0x1p-30);
    int l = 0;
    while (l < cap && std::ldexp(1.0, -(l + 1)) > k2) ++l;
    return l;
}

struct Problem {
    int model = 0;  // 0 GIRG, 1 HRG
    int64_t n = 0;
    int d = 1;
    double T = 0, K = 0, W = 0, w_min = 1, R = 0, alpha = 0;  // K: scale of Eq. 1
    uint64_t seed = 0;
    int precision = 0, edge_bytes = 4, level_cap = 0;
    const uint32_t* X = nullptr;  // d x n, original order
    const double* w = nullptr;    // original order
    const double* r = nullptr;    // HRG radii, original order
    Reduce red{};
};

// What the sampling rounds read, built from the points and the scale K: the layer
// partition and levels (host), and the sorted vertex arrays, cell offsets and bound
// tables (device).  Built by build_layout for every call, or kept by the resident
// point-set cache.
struct Layout {
    int L = 0, lcap = 0, m_int = 0, n3 = 1, n6 = 1, filt_k = 0;
    bool tzero = false;
    double invT = 0.0, coshR = 0.0;
    int64_t cnt[kMaxLayers] = {0};
    int I[kMaxLayers] = {0}, CLd[kMaxLayers] = {0};
    uint32_t layer_base[kMaxLayers + 1] = {0}, lstart[kMaxLayers + 1] = {0};
    std::vector<RowClass> classes;
    uint32_t *offs = nullptr, *skey = nullptr, *sid = nullptr, *Xs = nullptr;
    double* ws = nullptr;
    uint8_t* slayer = nullptr;
    float *sv = nullptr, *E32 = nullptr, *einv32 = nullptr, *sh32 = nullptr;
    uint4* vrec = nullptr;
    uint4* hrec = nullptr;
    TwoEntry* tii = nullptr;
    RowClass* d_classes = nullptr;
    uint8_t* jlist = nullptr;
    float *flo = nullptr, *fhi = nullptr;
};

// The edge buffer is device memory or page-locked host memory mapped into the
// device's address space (the kernels then write the edges across the host link, so
// no copy follows).  Pageable host memory is refused.
void* device_view(void* p) {
    if (!p) return p;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        throw Status{GIRG_E_PARAM};
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
    throw Status{GIRG_E_PARAM};
}

// Tables and sort (Sec. 3.1, 3.4, Lemma 1): fills Lo.  Buffers that Lo keeps come from
// A, temporaries from S (A may be S).  If order_out is set, stops after the sort and
// writes the sorted original ids there.
void build_layout(Problem& P, Scratch& A, Scratch& S, cudaStream_t st, Timer& tm, Layout& Lo,
                  int64_t* order_out) {
    const int64_t n = P.n;
    const int d = P.d;
    const bool girg = P.model == 0;
    const auto host_t0 = std::chrono::steady_clock::now();
    // ---------------------------------------------------------------- tables
    int L = 0;
    int64_t cnt[kMaxLayers];
    double wmax[kMaxLayers], rlo[kMaxLayers], rhi[kMaxLayers];
    for (int i = 0; i < kMaxLayers; ++i) {
        cnt[i] = (int64_t)P.red.cnt[i];
        wmax[i] = bits_to_double(P.red.wmax[i]);
        rlo[i] = bits_to_double(P.red.rmin[i]);
        rhi[i] = bits_to_double(P.red.rmax[i]);
        if (cnt[i]) L = i + 1;
    }
    int lcap = P.level_cap > 0 ? std::min(P.level_cap, 32 / d) : default_level_cap(n, d, P.T);
    const double invT = P.T > 0.0 ? 1.0 / P.T : 0.0;
    int m_int = 0;
    if (P.T > 0.0 && invT == std::floor(invT) && invT <= 64.0) m_int = (int)invT;
    double coshR = 0.0;
    if (!girg) {
        const double eR = det_exp(P.R);
        coshR = (eR + 1.0 / eR) * 0.5;
    }
    std::vector<std::vector<int>> CL(kMaxLayers, std::vector<int>(kMaxLayers, 0));
    int I[kMaxLayers] = {0}, CLd[kMaxLayers] = {0};
    for (int i = 0; i < L; ++i) {
        if (!cnt[i]) continue;
        for (int j = i; j < L; ++j) {
            if (!cnt[j]) continue;
            int cl;
            if (girg) {
                const double qmax = (wmax[i] * wmax[j]) / P.W;
                // the distance at which p reaches 1 (T > 0) or the threshold (T = 0)
                const double kappa = root_d(P.K * qmax, d);
                cl = level_for_kappa(kappa, lcap);
            } else {
                double gap = 0.0;
                if (rlo[j] > rhi[i]) gap = rlo[j] - rhi[i];
                if (rlo[i] > rhi[j]) gap = rlo[i] - rhi[j];
                const double eg = det_exp(gap);
                const double cg = (eg + 1.0 / eg) * 0.5;
                const double ei = det_exp(rlo[i]), ej = det_exp(rlo[j]);
                const double shi = (ei - 1.0 / ei) * 0.5, shj = (ej - 1.0 / ej) * 0.5;
                const double limit = coshR * (1.0 + 0x1p-30);
                cl = 1;
                while (cl < lcap) {
                    const double s = det_sinpi(std::ldexp(1.0, -(cl + 1)));
                    double t = shi * shj;
                    t = t * (s * s);
                    const double lb = cg + 2.0 * t;
                    if (!(lb > limit)) break;
                    ++cl;
                }
            }
            CL[i][j] = CL[j][i] = cl;
        }
    }
    for (int i = 0; i < L; ++i) {
        if (!cnt[i]) continue;
        for (int j = 0; j < L; ++j) {
            if (!cnt[j]) continue;
            I[i] = std::max(I[i], CL[i][j]);
            if (j >= i) CLd[i] = std::max(CLd[i], CL[i][j]);
        }
    }
    uint32_t layer_base[kMaxLayers + 1], lstart[kMaxLayers + 1];
    uint64_t total_cells = 0;
    for (int i = 0; i <= kMaxLayers; ++i) {
        if (total_cells >= 0xffffffffull) throw Status{GIRG_E_INTERNAL};
        layer_base[i] = (uint32_t)total_cells;
        if (i < L) total_cells += 1ull << (d * I[i]);
    }
    if (total_cells >= 0xfffffff0ull) throw Status{GIRG_E_INTERNAL};
    {
        uint64_t run = 0;
        for (int i = 0; i <= kMaxLayers; ++i) {
            lstart[i] = (uint32_t)run;
            if (i < kMaxLayers) run += (uint64_t)cnt[i];
        }
    }
    int n3 = 1, n6 = 1;
    for (int k = 0; k < d; ++k) {
        n3 *= 3;
        n6 *= 6;
    }
    const bool tzero = P.T == 0.0;
    double host_ms = host_ms_since(host_t0);
    tm.mark();  // layer partition done
    // ---------------------------------------------------------------- sort
    // the sorted keys and ids end up in two of these four (kept), the other two are free
    uint32_t* key = A.get<uint32_t>(n);
    uint32_t* val = A.get<uint32_t>(n);
    uint32_t* key2 = A.get<uint32_t>(2 * (size_t)n);  // one block: the placement's pairs
    uint32_t* val2 = key2 + n;
    uint32_t* offs = A.get<uint32_t>(total_cells + 1);
    uint32_t* stmp = S.get<uint32_t>(std::max({scan_tmp_words((int64_t)total_cells + 1),
                                               radix_tmp_words(n), place_tmp_words(n)}));
    CK(cudaMemsetAsync(offs, 0, (total_cells + 1) * sizeof(uint32_t), st));
    int8_t I8[kMaxLayers];
    for (int i = 0; i < kMaxLayers; ++i) I8[i] = (int8_t)I[i];
    const double* wsrc = P.w;
    // the order by placement, unless some layer averages more than 16 vertices a cell
    // (the large-cell sort would then carry much of the work): a stable radix sort
    // instead.  GIRG_SORT=radix or GIRG_SORT=place forces one (tests compare the two).
    bool place = true;
    for (int i = 0; i < L; ++i)
        if (cnt[i] > 0 && (uint64_t)cnt[i] > (16ull << (d * I[i]))) place = false;
    if (const char* env = std::getenv("GIRG_SORT")) {
        if (!std::strcmp(env, "radix")) place = false;
        if (!std::strcmp(env, "place")) place = true;
    }
    launch_keys(n, d, wsrc, P.X, girg ? P.w_min : 1.0, I8, layer_base, key, val, offs, place, st);
    launch_scan_u32(offs, offs, (int64_t)total_cells + 1, stmp, st);
    uint32_t *skey, *sid;
    if (place) {
        CK(cudaMemsetAsync(stmp, 0, sizeof(uint32_t), st));
        // the key-id pairs in key2 .. val2; the sorted keys and ids go to val and key
        place_by_counts(key, val, offs, n, reinterpret_cast<uint2*>(key2), val, key, stmp, st);
        skey = val;
        sid = key;
    } else {
        radix_sort_pairs(key, val, key2, val2, n, std::max(1, bitlen64(total_cells - 1)), stmp, st,
                         &skey, &sid);
    }
    if (order_out) {
        std::vector<uint32_t> h(n);
        CK(cudaMemcpyAsync(h.data(), sid, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::vector<int64_t> o(h.begin(), h.end());
        CK(cudaMemcpyAsync(order_out, o.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return;
    }
    // GIRG with d <= 4: packed vertex records (one or two 16-byte loads per vertex in the
    // pair tests); otherwise separate coordinate and scale arrays
    const bool packed = girg && d <= 4;
    uint32_t* Xs = packed ? nullptr : A.get<uint32_t>((size_t)d * n);
    double* ws = A.get<double>(n);
    uint8_t* slayer = A.get<uint8_t>(n);
    float *sv = nullptr, *E32 = nullptr, *einv32 = nullptr, *sh32 = nullptr;
    uint4 *vrec = nullptr, *hrec = nullptr;
    float gamma = 0.0f;
    const double log2W_half = girg ? 0.5 * std::log2(P.W) : 0.0;
    if (girg) {
        if (packed)
            vrec = A.get<uint4>((size_t)n * (d <= 2 ? 1 : 2));
        else
            sv = A.get<float>(n);
        gamma = (float)(std::log2(P.K) / (2.0 * d));  // kappa_uv = s_u s_v, kappa^d = K q
        launch_gather_girg(n, d, sid, P.X, P.w, P.w_min, log2W_half, gamma, (float)(1.0 / d), Xs,
                           ws, sv, slayer, vrec, st);
    } else {
        hrec = A.get<uint4>(n);  // angle, e^r, e^-r, sinh r of each sorted vertex
        launch_gather_hrg(n, sid, P.X, P.r, P.w, Xs, ws, E32, einv32, sh32, slayer, hrec, st);
    }
    tm.mark();  // sort done
    // the host tables of the sampler, built while the sort runs on the device
    const auto host_t1 = std::chrono::steady_clock::now();
    // row classes (i, l): the buckets j >= i with type II (CL >= l >= 2), then with
    // type I (CL = l)
    std::vector<RowClass> classes((size_t)std::max(L, 1) * (kMaxLevel + 1), RowClass{0, 0, 0});
    std::vector<uint8_t> jlist;
    for (int i = 0; i < L; ++i) {
        if (!cnt[i]) continue;
        for (int l = 0; l <= CLd[i]; ++l) {
            RowClass rc{0, 0, (uint32_t)jlist.size()};
            for (int j = i; j < L; ++j)
                if (cnt[j] && !tzero && l >= 2 && CL[i][j] >= l) {
                    jlist.push_back((uint8_t)j);
                    ++rc.n2;
                }
            for (int j = i; j < L; ++j)
                if (cnt[j] && CL[i][j] == l) {
                    jlist.push_back((uint8_t)j);
                    ++rc.n1;
                }
            classes[(size_t)i * (kMaxLevel + 1) + l] = rc;
        }
    }
    if (jlist.empty()) jlist.push_back(0);
    // type-II bounds for every (i <= j, l, g in {1, 2})
    std::vector<TwoEntry> tii((size_t)std::max(L, 1) * std::max(L, 1) * (lcap + 1) * 2);
    for (auto& e : tii) e = TwoEntry{0.0, 0.0, 0.0f, 0.0f, 62, 0};  // never read
    if (!tzero) {
        for (int i = 0; i < L; ++i) {
            if (!cnt[i]) continue;
            for (int j = i; j < L; ++j) {
                if (!cnt[j]) continue;
                for (int l = 2; l <= std::min(CL[i][j], lcap); ++l) {
                    for (int g = 1; g <= 2; ++g) {
                        double p;
                        if (girg) {
                            const double rmin = (double)g * std::ldexp(1.0, -l);
                            p = girg_p_at(wmax[i], wmax[j], rmin, P.W, P.K, invT, m_int, d);
                        } else {
                            double gap = 0.0;
                            if (rlo[j] > rhi[i]) gap = rlo[j] - rhi[i];
                            if (rlo[i] > rhi[j]) gap = rlo[i] - rhi[j];
                            const double eg = det_exp(gap);
                            const double cg = (eg + 1.0 / eg) * 0.5;
                            const double ei = det_exp(rlo[i]), ej = det_exp(rlo[j]);
                            const double shi = (ei - 1.0 / ei) * 0.5, shj = (ej - 1.0 / ej) * 0.5;
                            const double s = det_sinpi((double)g * std::ldexp(1.0, -l));
                            double t = shi * shj;
                            t = t * (s * s);
                            const double lb = cg + 2.0 * t;
                            p = hrg_p_from_coshd(lb, P.R, P.T);
                        }
                        p = p * (1.0 + 0x1p-30);
                        const double pbar = p < 1.0 ? p : 1.0;
                        TwoEntry e;
                        e.pbar = pbar;
                        e.Lb = pbar < 1.0 ? det_log1p(-pbar) : 0.0;
                        e.log2pbar = (float)std::log2(pbar);
                        e.invLb = pbar < 1.0 ? (float)(1.0 / e.Lb) : -INFINITY;
                        e.k = chunk_log(pbar);
                        e.one = pbar < 1.0 ? 0 : 1;
                        tii[((((size_t)i * L + j) * (lcap + 1) + l) << 1) + (g - 1)] = e;
                    }
                }
            }
        }
    }
    // HRG distance filter: thresholds on cosh d for U in bins of width 1/(K-1)
    const int K = 100;
    std::vector<float> flo(K, 1.0f), fhi(K, INFINITY);
    if (!girg && !tzero) {
        for (int m = 0; m < K; ++m) {
            const double x = (double)m / (double)(K - 1);
            double F;
            if (m == 0) {
                F = INFINITY;
            } else if (m == K - 1) {
                F = 1.0;
            } else {
                double pinv = P.R + 2.0 * P.T * std::log(1.0 / x - 1.0);
                if (pinv < 0.0) pinv = 0.0;
                F = std::cosh(pinv);
            }
            float f = (float)F;
            flo[m] = std::isinf(F) ? INFINITY : std::nextafterf(f, 0.0f) * (1.0f - 0x1p-22f);
            fhi[m] = std::isinf(F) ? INFINITY : std::nextafterf(f, INFINITY) * (1.0f + 0x1p-22f);
        }
    }
    host_ms += host_ms_since(host_t1);
    g_ms[9] = (float)host_ms;
    // ---------------------------------------------------------------- device tables
    TwoEntry* d_tii = A.get<TwoEntry>(tii.size());
    RowClass* d_classes = A.get<RowClass>(classes.size());
    uint8_t* d_jlist = A.get<uint8_t>(jlist.size());
    float* d_flo = A.get<float>(K);
    float* d_fhi = A.get<float>(K);
    CK(cudaMemcpyAsync(d_tii, tii.data(), tii.size() * sizeof(TwoEntry), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_classes, classes.data(), classes.size() * sizeof(RowClass),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_jlist, jlist.data(), jlist.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_flo, flo.data(), K * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_fhi, fhi.data(), K * 4, cudaMemcpyHostToDevice, st));
    // the host copies above read pageable vectors: they complete before the calls
    // return, so the vectors may go out of scope
    Lo.L = L;
    Lo.lcap = lcap;
    Lo.m_int = m_int;
    Lo.n3 = n3;
    Lo.n6 = n6;
    Lo.filt_k = K;
    Lo.tzero = tzero;
    Lo.invT = invT;
    Lo.coshR = coshR;
    for (int i = 0; i < kMaxLayers; ++i) {
        Lo.cnt[i] = cnt[i];
        Lo.I[i] = I[i];
        Lo.CLd[i] = CLd[i];
    }
    memcpy(Lo.layer_base, layer_base, sizeof(layer_base));
    memcpy(Lo.lstart, lstart, sizeof(lstart));
    Lo.classes = std::move(classes);
    Lo.offs = offs;
    Lo.skey = skey;
    Lo.sid = sid;
    Lo.Xs = Xs;
    Lo.ws = ws;
    Lo.slayer = slayer;
    Lo.sv = sv;
    Lo.E32 = E32;
    Lo.einv32 = einv32;
    Lo.sh32 = sh32;
    Lo.vrec = vrec;
    Lo.hrec = hrec;
    Lo.tii = d_tii;
    Lo.d_classes = d_classes;
    Lo.jlist = d_jlist;
    Lo.flo = d_flo;
    Lo.fhi = d_fhi;
}

// Cell-pair enumeration and sampling (Algorithm 1, Sec. 3.2, 3.3) over a layout: rows,
// work lists in rounds, type I and type II, edge count and statistics.
void run_sampler(Problem& P, const Layout& Lo, Scratch& S, cudaStream_t st, Timer& tm,
                 void* d_edges, int64_t cap, int64_t* num_edges) {
    d_edges = device_view(d_edges);
    const int64_t n = P.n;
    const int d = P.d;
    const bool girg = P.model == 0;
    const int L = Lo.L, lcap = Lo.lcap, m_int = Lo.m_int, n3 = Lo.n3, n6 = Lo.n6, K = Lo.filt_k;
    const bool tzero = Lo.tzero;
    const double invT = Lo.invT, coshR = Lo.coshR;
    const int64_t* cnt = Lo.cnt;
    const int *I = Lo.I, *CLd = Lo.CLd;
    const std::vector<RowClass>& classes = Lo.classes;
    uint32_t *offs = Lo.offs, *skey = Lo.skey, *sid = Lo.sid, *Xs = Lo.Xs;
    double* ws = Lo.ws;
    uint8_t* slayer = Lo.slayer;
    float *sv = Lo.sv, *E32 = Lo.E32, *einv32 = Lo.einv32, *sh32 = Lo.sh32;
    uint4* vrec = Lo.vrec;
    TwoEntry* d_tii = Lo.tii;
    RowClass* d_classes = Lo.d_classes;
    uint8_t* d_jlist = Lo.jlist;
    float *d_flo = Lo.flo, *d_fhi = Lo.fhi;
    // work entries: at most min(|V_i|, 2^(d l)) rows per (i, l), one entry per bucket
    uint64_t ent2_cap = 0, ent1_cap = 0;
    for (int i = 0; i < L; ++i)
        for (int l = 0; l <= CLd[i] && cnt[i]; ++l) {
            const uint64_t rows_il =
                std::min<uint64_t>((uint64_t)cnt[i], d * l >= 63 ? ~0ull : (1ull << (d * l)));
            const RowClass& rc = classes[(size_t)i * (kMaxLevel + 1) + l];
            ent2_cap += rows_il * rc.n2;
            ent1_cap += rows_il * rc.n1;
        }
    if (ent2_cap >= 0xffffffffull || ent1_cap >= 0xffffffffull) throw Status{GIRG_E_INTERNAL};
    uint64_t* ent2 = S.get<uint64_t>(ent2_cap + 1);
    uint64_t* ent1 = S.get<uint64_t>(ent1_cap + 1);
    // the small counters in one block, cleared with one memset: stats (then the edge
    // count and the two work counters of the type-I / type-II kernels), one round's
    // work-list counts (type-I items, streams, segments) and statistics, and the 32-bit
    // row / entry / error counters
    constexpr size_t kSmallWords = kNumStats + 3 + 3 + kNumStats + 8;
    unsigned long long* small = S.get<unsigned long long>(kSmallWords);
    unsigned long long* stats = small;
    unsigned long long* wcount = stats + kNumStats + 3;
    unsigned long long* estats = wcount + 3;
    unsigned int* counters = reinterpret_cast<unsigned int*>(estats + kNumStats);
    CK(cudaMemsetAsync(small, 0, kSmallWords * sizeof(unsigned long long), st));
    // work lists, sized from typical counts per vertex; the enumeration only writes
    // work (no edges), so an overflow is repaired by resizing and running it again
    // GIRG_INITIAL_LIST_SCALE in (0, 1] shrinks the initial sizes (tests use it to
    // drive the overflow, growth and rerun paths at small n)
    double list_scale = 1.0;
    if (const char* env = std::getenv("GIRG_INITIAL_LIST_SCALE")) {
        const double v = std::atof(env);
        if (v > 0.0 && v <= 1.0) list_scale = v;
    }
    auto clamp_cap = [list_scale](uint64_t c, uint64_t mx) {
        c = (uint64_t)((double)c * list_scale);
        c = c < 16 ? 16 : c;
        return c > mx ? mx : c;
    };
    // estimated list sizes at or beyond the maxima of one round: the first round would
    // overflow, so it only counts (the rounds below are planned from its counts)
    const uint64_t est_t1 = (uint64_t)n * (1 + (uint64_t)(0.75 * n3)) + 65536;
    uint64_t t1_cap = clamp_cap(est_t1, 1ull << 30);
    uint64_t stream_cap =
        tzero ? 1024 : clamp_cap((uint64_t)n * (2 + 2 * (uint64_t)d) + 65536, 1ull << 28);
    // partner segments per vertex measured at n = 10^6, beta = 2.2, T = 0.7: about 4.3,
    // 19, 81 and 325 for d = 1..4 (they grow like 6^d); sized with headroom
    const uint64_t seg_per_v = d == 1 ? 8 : d == 2 ? 28 : d == 3 ? 112 : d == 4 ? 448 : 4 * (uint64_t)n6;
    const uint64_t est_seg = (uint64_t)n * seg_per_v + 65536;
    uint64_t seg_cap = tzero ? 1024 : clamp_cap(est_seg, 1ull << 31);
    bool count_first = list_scale == 1.0 && (est_t1 > (1ull << 30) || (!tzero && est_seg > (1ull << 31)));
    // GIRG_COUNT_FIRST=1 forces it (tests drive that path at small n with shrunk lists)
    if (const char* env = std::getenv("GIRG_COUNT_FIRST")) count_first = env[0] == '1';
    T1Item* t1 = S.get<T1Item>(t1_cap);
    uint32_t* t1_pairs = S.get<uint32_t>(t1_cap + 1);
    Stream* streams = S.get<Stream>(stream_cap);
    uint32_t* stream_chunks = S.get<uint32_t>(stream_cap + 1);
    Seg* segs = S.get<Seg>(seg_cap);

    DevCfg cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.n = (int32_t)n;
    cfg.d = d;
    cfg.L = L;
    cfg.model = P.model;
    cfg.precision = P.precision;
    cfg.tzero = tzero ? 1 : 0;
    cfg.m_int = m_int;
    cfg.lcap = lcap;
    cfg.n3 = n3;
    cfg.n6 = n6;
    cfg.seed_lo = (uint32_t)P.seed;
    cfg.seed_hi = (uint32_t)(P.seed >> 32);
    cfg.W = P.W;
    cfg.K = P.K;
    cfg.T = P.T;
    cfg.invT = invT;
    cfg.w_min = P.w_min;
    cfg.R = P.R;
    cfg.coshR = coshR;
    cfg.dT = P.T > 0.0 ? (float)(d / P.T) : 0.0f;
    if (girg)
        cfg.bandG = cfg.dT * 0x1p-14f + 0x1p-15f;
    else
        cfg.bandG = (float)(0x1p-12 * (1.0 + (P.T > 0.0 ? 0.5 / P.T : 0.0)));
    cfg.band_ratio = 0x1p-16f;
    cfg.coshR32 = (float)coshR;
    cfg.R32 = (float)P.R;
    cfg.inv2T32 = P.T > 0.0 ? (float)(0.5 / P.T) : 0.0f;
    cfg.filt_k = K;
    for (int i = 0; i < kMaxLayers; ++i) {
        cfg.I[i] = (int8_t)I[i];
        cfg.CLd[i] = (uint8_t)CLd[i];
    }
    memcpy(cfg.layer_base, Lo.layer_base, sizeof(Lo.layer_base));
    memcpy(cfg.lstart, Lo.lstart, sizeof(Lo.lstart));
    cfg.tii = d_tii;
    cfg.classes = d_classes;
    cfg.jlist = d_jlist;
    cfg.offs = offs;
    cfg.Xs = Xs;
    cfg.sv = sv;
    cfg.ws = ws;
    cfg.ids = sid;
    cfg.skey = skey;
    cfg.slayer = slayer;
    cfg.E32 = E32;
    cfg.einv32 = einv32;
    cfg.sh32 = sh32;
    cfg.hrec = Lo.hrec;
    cfg.vrec = vrec;
    cfg.filt_lo = d_flo;
    cfg.filt_hi = d_fhi;
    cfg.edges = d_edges;
    cfg.edge_bytes = P.edge_bytes;
    cfg.cap = P.edge_bytes == 0 ? INT64_MAX : cap;  // count-only: nothing is stored
    cfg.edge_count = stats + kNumStats;
    cfg.stats = stats;
    cfg.row_count = counters + 0;
    cfg.ent2 = ent2;
    cfg.ent2_count = counters + 6;
    cfg.ent2_cap = (uint32_t)ent2_cap;
    cfg.ent1 = ent1;
    cfg.ent1_count = counters + 7;
    cfg.ent1_cap = (uint32_t)ent1_cap;
    cfg.t1 = t1;
    cfg.t1_count = wcount + 0;
    cfg.t1_cap = (uint32_t)t1_cap;
    cfg.t1_pairs = t1_pairs;
    cfg.streams = streams;
    cfg.stream_count = wcount + 1;
    cfg.stream_cap = (uint32_t)stream_cap;
    cfg.stream_chunks = stream_chunks;
    cfg.segs = segs;
    cfg.seg_count = wcount + 2;
    cfg.seg_cap = (uint32_t)seg_cap;
    cfg.error = counters + 5;
    cfg.work64 = stats + kNumStats + 1;

    launch_rows(cfg, st);
    // Enumeration and sampling in rounds over ranges of the work entries: a round's
    // lists must fit their capacities (grown up to a maximum); a round whose lists
    // would exceed the maximum is retried over fewer entries.  The enumeration writes
    // no edges, so a retried round leaves no trace (its statistics are kept apart
    // until it is accepted).
    constexpr uint64_t kMaxT1 = 1ull << 30, kMaxStreams = 1ull << 28, kMaxSegs = 1ull << 31;
    uint32_t lo2 = 0, lo1 = 0, hi2 = 0xffffffffu, hi1 = 0xffffffffu;
    unsigned long long est_acc[kNumStats] = {0};
    uint64_t total_streams = 0, total_segs = 0, passes = 0, n_ent2 = 0, n_ent1 = 0;
    unsigned long long *t1_pre = nullptr, *chunk_pre = nullptr, *tmp = nullptr;
    size_t pre_cap1 = 0, pre_cap2 = 0, tmp_cap = 0;
    int round = 0;
    unsigned long long hs[kNumStats + 1];
    unsigned int rc[6];
    // The first round runs without a host round trip: the scans take the list
    // lengths from the device and the counts are checked afterwards, read back with
    // the statistics.  If a list overflowed, the round is undone (statistics and
    // edge count restored from a copy; the edges it wrote are overwritten later) and
    // the rounds below take over.
    bool done = false;
    // the list counts of an overflowed first round: the first attempt below would run
    // the same enumeration again, so it starts from these instead
    bool have_first = false;
    unsigned long long first_wc[3] = {0, 0, 0};
    unsigned int first_ec[2] = {0, 0};
    if (count_first) {  // entries, lists and statistics counted, nothing written
        cfg.ent2_lo = 0;
        cfg.ent2_hi = 0xffffffffu;
        cfg.ent1_lo = 0;
        cfg.ent1_hi = 0xffffffffu;
        DevCfg ecfg = cfg;
        ecfg.stats = estats;
        ecfg.count_only = 1;
        launch_enumerate(ecfg, st);
        ++passes;
        unsigned long long wc[3];
        unsigned int ec[2];
        CK(cudaMemcpyAsync(wc, wcount, sizeof(wc), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ec, counters + 6, sizeof(ec), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        n_ent2 = ec[0];
        n_ent1 = ec[1];
        if (wc[0] > cfg.t1_cap || wc[1] > cfg.stream_cap || wc[2] > cfg.seg_cap) {
            memcpy(first_wc, wc, sizeof(wc));
            memcpy(first_ec, ec, sizeof(ec));
            have_first = true;
        }  // else the rounds below enumerate again, writing
    } else {
        cfg.ent2_lo = 0;
        cfg.ent2_hi = 0xffffffffu;
        cfg.ent1_lo = 0;
        cfg.ent1_hi = 0xffffffffu;  // wcount and estats are clear from the block memset
        DevCfg ecfg = cfg;
        ecfg.stats = estats;
        launch_enumerate(ecfg, st);
        ++passes;
        pre_cap1 = cfg.t1_cap + 1ull;
        pre_cap2 = cfg.stream_cap + 1ull;
        t1_pre = S.get<unsigned long long>(pre_cap1);
        chunk_pre = S.get<unsigned long long>(pre_cap2);
        tmp_cap = scan_tmp_words((int64_t)std::max(pre_cap1, pre_cap2));
        tmp = S.get<unsigned long long>(tmp_cap);
        unsigned long long* lens = S.get<unsigned long long>(2);
        unsigned int* ok = S.get<unsigned int>(1);
        unsigned long long* snap = S.get<unsigned long long>(kNumStats + 3);
        CK(cudaMemcpyAsync(snap, stats, (kNumStats + 3) * sizeof(unsigned long long),
                           cudaMemcpyDeviceToDevice, st));
        launch_prep_lists(cfg, lens, ok, st);
        cfg.lists_ok = ok;  // an overflowed round samples nothing
        launch_scan_u32_to_u64_dev(cfg.t1_pairs, t1_pre, lens, (int64_t)pre_cap1, tmp, st);
        launch_scan_u32_to_u64_dev(cfg.stream_chunks, chunk_pre, lens + 1, (int64_t)pre_cap2, tmp, st);
        cfg.t1_pre = t1_pre;
        cfg.chunk_pre = chunk_pre;
        tm.mark();  // enumeration and its list scans done
        launch_type1(cfg, st);
        tm.mark();  // type I done
        launch_type2(cfg, st);
        tm.mark();  // type II done
        cfg.lists_ok = nullptr;  // the rounds below check the counts on the host first
        // the whole counter block in one readback: statistics and edge count, the
        // round's list counts and statistics, the row / entry / error counters
        unsigned long long hsmall[kSmallWords];
        CK(cudaMemcpyAsync(hsmall, small, sizeof(hsmall), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        unsigned long long wc[3], es[kNumStats];
        unsigned int ec[2];
        memcpy(wc, hsmall + (wcount - small), sizeof(wc));
        memcpy(es, hsmall + (estats - small), sizeof(es));
        memcpy(hs, hsmall + (stats - small), sizeof(hs));
        const unsigned char* hcounters =
            reinterpret_cast<const unsigned char*>(hsmall + (estats + kNumStats - small));
        memcpy(rc, hcounters, sizeof(rc));
        memcpy(ec, hcounters + 6 * sizeof(unsigned int), sizeof(ec));
        n_ent2 = ec[0];
        n_ent1 = ec[1];
        if (wc[0] <= cfg.t1_cap && wc[1] <= cfg.stream_cap && wc[2] <= cfg.seg_cap) {
            for (int q = 0; q < kNumStats; ++q) est_acc[q] += es[q];
            total_streams += wc[1];
            total_segs += wc[2];
            round = 1;
            done = true;
        } else {
            CK(cudaMemcpyAsync(stats, snap, (kNumStats + 3) * sizeof(unsigned long long),
                               cudaMemcpyDeviceToDevice, st));
            tm.used -= 3;  // the rounds below mark these phases again
            memcpy(first_wc, wc, sizeof(wc));
            memcpy(first_ec, ec, sizeof(ec));
            have_first = true;
        }
    }
    for (int attempt = 0; !done; ++attempt) {
        if (attempt > 64) throw Status{GIRG_E_INTERNAL};
        cfg.ent2_lo = lo2;
        cfg.ent2_hi = hi2;
        cfg.ent1_lo = lo1;
        cfg.ent1_hi = hi1;
        unsigned long long wc[3], es[kNumStats];
        unsigned int ec[2];
        if (have_first) {  // same entries and capacities as the first round: its counts
            have_first = false;
            memcpy(wc, first_wc, sizeof(wc));
            memcpy(ec, first_ec, sizeof(ec));
            memset(es, 0, sizeof(es));  // unused: these counts overflow
        } else {
            CK(cudaMemsetAsync(wcount, 0, 3 * sizeof(unsigned long long), st));
            CK(cudaMemsetAsync(estats, 0, kNumStats * sizeof(unsigned long long), st));
            DevCfg ecfg = cfg;
            ecfg.stats = estats;
            launch_enumerate(ecfg, st);
            ++passes;
            CK(cudaMemcpyAsync(wc, wcount, sizeof(wc), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(ec, counters + 6, sizeof(ec), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(es, estats, sizeof(es), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
        const uint32_t e2 = std::min<uint32_t>(ec[0], cfg.ent2_cap);
        const uint32_t e1 = std::min<uint32_t>(ec[1], cfg.ent1_cap);
        const uint32_t end2 = std::min(hi2, e2), end1 = std::min(hi1, e1);
        n_ent2 = ec[0];
        n_ent1 = ec[1];
        if (wc[0] > cfg.t1_cap || wc[1] > cfg.stream_cap || wc[2] > cfg.seg_cap) {
            double f = 1.0;
            if (wc[0] > kMaxT1) f = std::min(f, 0.8 * (double)kMaxT1 / (double)wc[0]);
            if (wc[1] > kMaxStreams) f = std::min(f, 0.8 * (double)kMaxStreams / (double)wc[1]);
            if (wc[2] > kMaxSegs) f = std::min(f, 0.8 * (double)kMaxSegs / (double)wc[2]);
            if (f < 1.0) {  // fewer entries this round
                hi2 = lo2 + std::max<uint32_t>(1, (uint32_t)((end2 - lo2) * f));
                hi1 = lo1 + std::max<uint32_t>(1, (uint32_t)((end1 - lo1) * f));
                continue;
            }
            if (wc[0] > cfg.t1_cap) {
                cfg.t1_cap = (uint32_t)std::min<uint64_t>(kMaxT1, wc[0] + wc[0] / 16 + 1024);
                cfg.t1 = S.get<T1Item>(cfg.t1_cap);
                cfg.t1_pairs = S.get<uint32_t>((size_t)cfg.t1_cap + 1);
            }
            if (wc[1] > cfg.stream_cap) {
                cfg.stream_cap = (uint32_t)std::min<uint64_t>(kMaxStreams, wc[1] + wc[1] / 16 + 1024);
                cfg.streams = S.get<Stream>(cfg.stream_cap);
                cfg.stream_chunks = S.get<uint32_t>((size_t)cfg.stream_cap + 1);
            }
            if (wc[2] > cfg.seg_cap) {
                cfg.seg_cap = (uint32_t)std::min<uint64_t>(kMaxSegs, wc[2] + wc[2] / 16 + 1024);
                cfg.segs = S.get<Seg>(cfg.seg_cap);
            }
            continue;
        }
        for (int q = 0; q < kNumStats; ++q) est_acc[q] += es[q];
        // exclusive prefixes of the pairs per type-I item and of the chunks per stream
        // (one past the last entry holds the total)
        const uint32_t n1 = (uint32_t)wc[0], ns = (uint32_t)wc[1];
        total_streams += ns;
        total_segs += wc[2];
        if (n1 + 1ull > pre_cap1) {  // prefix buffers, reused by later rounds
            pre_cap1 = n1 + 1ull + (n1 >> 3);
            t1_pre = S.get<unsigned long long>(pre_cap1);
        }
        if (ns + 1ull > pre_cap2) {
            pre_cap2 = ns + 1ull + (ns >> 3);
            chunk_pre = S.get<unsigned long long>(pre_cap2);
        }
        const size_t tw = scan_tmp_words((int64_t)std::max(pre_cap1, pre_cap2));
        if (tw > tmp_cap) {
            tmp_cap = tw;
            tmp = S.get<unsigned long long>(tmp_cap);
        }
        CK(cudaMemsetAsync(cfg.t1_pairs + n1, 0, sizeof(uint32_t), st));
        CK(cudaMemsetAsync(cfg.stream_chunks + ns, 0, sizeof(uint32_t), st));
        CK(cudaMemsetAsync(cfg.work64, 0, 2 * sizeof(unsigned long long), st));
        launch_scan_u32_to_u64(cfg.t1_pairs, t1_pre, (int64_t)n1 + 1, tmp, st);
        launch_scan_u32_to_u64(cfg.stream_chunks, chunk_pre, (int64_t)ns + 1, tmp, st);
        cfg.t1_pre = t1_pre;
        cfg.chunk_pre = chunk_pre;
        if (round == 0) tm.mark();  // (first round) enumeration and list scans done
        launch_type1(cfg, st);
        if (round == 0) tm.mark();  // (first round) type I done
        launch_type2(cfg, st);
        ++round;
        if (end2 >= e2 && end1 >= e1) break;
        // the next round: as many entries as this one
        const uint32_t span2 = end2 - lo2, span1 = end1 - lo1;
        lo2 = end2;
        lo1 = end1;
        hi2 = (uint32_t)std::min<uint64_t>(0xffffffffull, (uint64_t)lo2 + std::max<uint32_t>(span2, 1));
        hi1 = (uint32_t)std::min<uint64_t>(0xffffffffull, (uint64_t)lo1 + std::max<uint32_t>(span1, 1));
        attempt = 0;
    }
    if (!done) {
        tm.mark();  // type II done (with every later round)
        CK(cudaMemcpyAsync(hs, stats, (kNumStats + 1) * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(rc, counters, 6 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    CK(cudaGetLastError());
    if (rc[5]) throw Status{GIRG_E_INTERNAL};
    for (int q = 0; q < kNumStats; ++q) hs[q] += est_acc[q];
    hs[kStatRows] = rc[0];
    hs[kStatEdges] = hs[kNumStats];
    hs[kStatStreams] = total_streams;
    hs[kStatSegs] = total_segs;
    hs[kStatEnumPasses] = passes;
    hs[kStatEnt2] = n_ent2;
    hs[kStatEnt1] = n_ent1;
    for (int q = 0; q < kNumStats; ++q) g_stats[q] = (int64_t)hs[q];
    g_stats[kStatLaunches] = (int64_t)g_launches;
    *num_edges = (int64_t)hs[kNumStats];
}

void finish_timing(Timer& tm) {
    for (int q = 0; q < 7; ++q) g_ms[q] = 0.0f;
    // marks: 0 start, 1 reduce done, 2 layer partition, 3 sort, 4 enumerate, 5 type I, 6 type II
    for (int q = 1; q < tm.used && q <= 6; ++q) cudaEventElapsedTime(&g_ms[q - 1], tm.ev[q - 1], tm.ev[q]);
    if (tm.used >= 2) cudaEventElapsedTime(&g_ms[6], tm.ev[0], tm.ev[tm.used - 1]);
}

void read_reduce(Problem& P, Reduce* d_red, cudaStream_t st) {
    CK(cudaMemcpyAsync(&P.red, d_red, sizeof(Reduce), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
}

Reduce* new_reduce(Scratch& S, cudaStream_t st) {
    Reduce* red = S.get<Reduce>(1);
    CK(cudaMemsetAsync(red, 0, sizeof(Reduce), st));
    CK(cudaMemsetAsync(red->rmin, 0xff, sizeof(red->rmin), st));
    return red;
}

int exponent_of_ulp(double w) {  // every double >= w is an integer multiple of 2^E0
    int e;
    std::frexp(w, &e);
    return e - 53;
}

int check_girg(const girg_params* p) {
    if (!p) return GIRG_E_PARAM;
    if (p->n < 2 || p->n >= (1ll << 31)) return GIRG_E_PARAM;
    if (p->d < 1 || p->d > kMaxDim) return GIRG_E_PARAM;
    if (!(p->beta > 2.0) || !(p->T >= 0.0 && p->T < 1.0) || !(p->w_min > 0.0)) return GIRG_E_PARAM;
    if (p->edge_bytes != 0 && p->edge_bytes != 4 && p->edge_bytes != 8) return GIRG_E_PARAM;
    if (p->precision != 0 && p->precision != 1) return GIRG_E_PARAM;
    if (!(p->c > 0.0) && !(p->avg_deg > 0.0 && p->avg_deg < (double)(p->n - 1))) return GIRG_E_PARAM;
    if (p->level_cap < 0) return GIRG_E_PARAM;
    return GIRG_OK;
}

template <class F>
int guarded(F&& f) {
    try {
        if (!det_tables_gen() || !det_tables_pairs()) return GIRG_E_CUDA;
        return f();
    } catch (const CudaFail& e) {
        fprintf(stderr, "girg_gb300: CUDA error %s\n", cudaGetErrorString(e.err));
        return GIRG_E_CUDA;
    } catch (const Status& s) {
        return s.code;
    } catch (const std::bad_alloc&) {
        return GIRG_E_INTERNAL;
    } catch (const std::exception& e) {  // e.g. a host thread that could not start
        fprintf(stderr, "girg_gb300: %s\n", e.what());
        return GIRG_E_INTERNAL;
    }
}

// Host copy of a weight split (pinned, one per host thread, kept for the life of the
// process): the weights above thr (sorted on the device when there are at most
// kTopSortMax of them) and the four sums over the rest.
struct SplitHost {
    unsigned int count[2];  // gathered, sorted flag
    double thr;
    double sums[4];         // sum w, sum w^2, sum (w/thr)^(1/T), sum (w/thr)^(2/T)
    double w[kTopSortMax];
};

SplitHost* pinned_split() {
    thread_local SplitHost* p = nullptr;
    if (!p) {
        void* q = nullptr;
        CK(cudaMallocHost(&q, sizeof(SplitHost)));
        p = static_cast<SplitHost*>(q);
    }
    return p;
}

// Device buffers of the weight split.
struct SplitDev {
    unsigned int* cnt;
    double *thr, *sums, *part, *buf, *sorted;
    unsigned int cap;
};

SplitDev split_buffers(int64_t n, Scratch& S) {
    SplitDev D;
    D.cnt = S.get<unsigned int>(3);  // gathered, sorted flag, blocks done
    D.thr = S.get<double>(1);
    D.sums = S.get<double>(4);
    D.part = S.get<double>((size_t)4 * reduce_blocks(n));
    // more than the one-block sort takes: a radix sort orders those; sized so that the
    // split rarely has to run a second time with a larger buffer
    D.cap = (unsigned int)std::max<int64_t>(4 * kTopSortMax, n / 32);
    D.buf = S.get<double>(D.cap);
    D.sorted = S.get<double>(kTopSortMax);
    return D;
}

// Queue the split at the threshold in D.thr and the copy of its results into h
// (read after the next synchronisation).
void queue_split(const Problem& P, SplitDev& D, SplitHost* h, cudaStream_t st) {
    CK(cudaMemsetAsync(D.cnt, 0, 3 * sizeof(unsigned int), st));
    launch_split_weights(P.n, P.w, D.thr, P.T, D.buf, D.cap, D.cnt, D.part, D.sums, D.sorted, st);
    CK(cudaMemcpyAsync(h->count, D.cnt, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&h->thr, D.thr, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->sums, D.sums, sizeof(h->sums), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->w, D.sorted, sizeof(h->w), cudaMemcpyDeviceToHost, st));
}

// Hand a finished split to the degree model; when more weights were gathered than the
// one-block sort takes, a device radix sort orders them before the copy (the buffer is
// enlarged and the split rerun when they did not fit).
void take_split(const Problem& P, DegreeModel& M, SplitDev& D, SplitHost* h, Scratch& S,
                cudaStream_t st) {
    unsigned int k = h->count[0];
    if (h->count[1] == 1u) {
        M.set_split(h->thr, std::vector<double>(h->w, h->w + k), h->sums[0], h->sums[1],
                    h->sums[2], h->sums[3]);
        return;
    }
    if (k > D.cap) {
        D.cap = k + 1024;
        D.buf = S.get<double>(D.cap);
        queue_split(P, D, h, st);
        CK(cudaStreamSynchronize(st));
        k = h->count[0];
    }
    std::vector<double> top(k);
    if (k) {
        double* sorted = S.get<double>(k);
        sort_f64_desc(D.buf, k, sorted, S.get<uint32_t>(sort_desc_words(k)), st);
        CK(cudaMemcpyAsync(top.data(), sorted, k * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    M.set_split(h->thr, std::move(top), h->sums[0], h->sums[1], h->sums[2], h->sums[3]);
}

// Solve the scale K for the target degree from the split queued with the reduction;
// a new split at a lower threshold is made only if the search needs it.
double solve_K(Problem& P, double target, SplitDev& D, SplitHost* h, Scratch& S,
               cudaStream_t st) {
    DegreeModel M(P.n, P.d, P.T, P.W);
    take_split(P, M, D, h, S, st);
    auto fetch = [&](double thr) {
        CK(cudaMemcpyAsync(D.thr, &thr, sizeof(double), cudaMemcpyHostToDevice, st));
        queue_split(P, D, h, st);
        CK(cudaStreamSynchronize(st));
        take_split(P, M, D, h, S, st);
    };
    return M.solve(target, fetch);
}

// The c of Eq. 1 for a scale K (0 or inf where it leaves the range of doubles).
double c_of_K(double K, int d, double T) {
    const double e = std::log(K) / (T > 0.0 ? T : (double)d);
    return e < -745.0 ? 0.0 : (e > 709.0 ? INFINITY : std::exp(e));
}

thread_local double g_last_K = 0.0;

// The reservation of a generate call's scratch: the server's admission estimate, an
// upper bound of what the call takes at its initial work-list sizes.
size_t scratch_reserve(const girg_params& p) {
    const int64_t b = girg_scratch_bytes(&p);
    return b > 0 ? (size_t)b : 0;
}

// ------------------------------------------------------------------ resident point sets
// With the cache on (girg_point_cache), girg_generate keeps the layout of each graph it
// builds -- sorted vertex arrays, cell offsets, bound tables, levels -- on the device,
// keyed by every input the layout depends on: the points (n, d, beta, w_min, seed), the
// scale (T with c, or with the target degree) and the level cap.  A call with the same
// values samples from the kept layout and makes the same graph.  Entries are evicted
// least recently used first beyond the byte limit; an entry in use by a call is freed
// when that call releases it (every call has synchronised its stream by then).
struct CacheKey {
    int64_t n;
    int d, level_cap, dev;
    double beta, w_min, T, c, avg_deg;
    uint64_t seed;
    bool operator==(const CacheKey& o) const {
        return n == o.n && d == o.d && level_cap == o.level_cap && dev == o.dev &&
               beta == o.beta && w_min == o.w_min && T == o.T && c == o.c &&
               avg_deg == o.avg_deg && seed == o.seed;
    }
};

struct CacheEntry {
    CacheKey key;
    Layout Lo;
    double K = 0.0, W = 0.0, w_min = 0.0, c_used = 0.0;
    std::vector<void*> bufs;
    size_t bytes = 0;
    uint64_t last_use = 0;
    ~CacheEntry() {  // on the entry's device; the calling thread's device is restored
        int prev = 0;
        const bool switch_dev = cudaGetDevice(&prev) == cudaSuccess && prev != key.dev;
        if (switch_dev) cudaSetDevice(key.dev);
        for (void* p : bufs) cudaFree(p);
        if (switch_dev) cudaSetDevice(prev);
    }
};

struct PointCache {
    std::mutex mu;
    int64_t max_bytes = 0;  // 0: off
    int64_t bytes = 0, hits = 0, misses = 0;
    uint64_t clock = 0;
    std::vector<std::shared_ptr<CacheEntry>> entries;

    std::shared_ptr<CacheEntry> find(const CacheKey& k) {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& e : entries)
            if (e->key == k) {
                e->last_use = ++clock;
                ++hits;
                return e;
            }
        ++misses;
        return nullptr;
    }
    // Keep e unless an equal entry arrived meanwhile or it alone exceeds the limit;
    // evict least recently used entries beyond the limit.
    void insert(std::shared_ptr<CacheEntry> e) {
        std::lock_guard<std::mutex> lk(mu);
        if (max_bytes <= 0 || (int64_t)e->bytes > max_bytes) return;
        for (auto& x : entries)
            if (x->key == e->key) return;
        e->last_use = ++clock;
        bytes += (int64_t)e->bytes;
        entries.push_back(std::move(e));
        while (bytes > max_bytes && !entries.empty()) {
            size_t oldest = 0;
            for (size_t i = 1; i < entries.size(); ++i)
                if (entries[i]->last_use < entries[oldest]->last_use) oldest = i;
            bytes -= (int64_t)entries[oldest]->bytes;
            entries.erase(entries.begin() + (long)oldest);
        }
    }
};

PointCache& point_cache() {
    static PointCache* c = new PointCache();  // never destroyed: no CUDA calls at exit
    return *c;
}

bool cache_on() {
    PointCache& c = point_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    return c.max_bytes > 0;
}

}  // namespace

extern "C" {

const char* girg_status_string(int status) {
    switch (status) {
        case GIRG_OK: return "ok";
        case GIRG_E_PARAM: return "parameter out of range";
        case GIRG_E_CAPACITY: return "edge buffer too small";
        case GIRG_E_CUDA: return "CUDA error";
        case GIRG_E_RANGE: return "weights span too wide a range for the exact sum";
        case GIRG_E_INTERNAL: return "internal capacity or consistency check failed";
        default: return "unknown status";
    }
}

double girg_det_eval(int32_t fn, double x, double y) {
    switch (fn) {
        case 0: return det_log(x);
        case 1: return det_log1p(x);
        case 2: return det_exp(x);
        case 3: return det_pow(x, y);
        case 4: return det_sinpi(x);
        case 5: return det_acosh(x);
        case 6: return girg_p_at(x, y, 0.25, 1000.0, girg_K_of_c(0.5, 2, 0.75), 1.0 / 0.75, 0, 2);
        case 7: return (double)layer_of_bits(x, y);
        default: return dnan();
    }
}

int64_t girg_expected_edges(const girg_params* params, void* stream) {
    if (!params) return -1;
    if (params->c > 0.0) {
        double f = 0.0;
        if (girg_expected_avg_degree(params, &f, stream) != GIRG_OK) return -1;
        return (int64_t)std::llround(0.5 * f * (double)params->n);
    }
    // solved c: the expected degree is the target by construction
    if (check_girg(params) != GIRG_OK) return -1;
    return (int64_t)std::llround(0.5 * params->avg_deg * (double)params->n);
}

double girg_last_scale(void) { return g_last_K; }

int girg_scratch_pool_usage(int64_t* reserved, int64_t* used, int64_t* used_high,
                            int32_t reset_high) {
    return guarded([&] {
        cudaMemPool_t pool = library_pool();
        uint64_t v = 0;
        if (reserved) {
            CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v));
            *reserved = (int64_t)v;
        }
        if (used) {
            CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v));
            *used = (int64_t)v;
        }
        if (used_high) {
            CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v));
            *used_high = (int64_t)v;
        }
        if (reset_high) {
            uint64_t zero = 0;
            CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
        }
        return GIRG_OK;
    });
}

int girg_point_cache(int64_t max_bytes) {
    if (max_bytes < 0) return GIRG_E_PARAM;
    std::vector<std::shared_ptr<CacheEntry>> drop;
    {
        PointCache& c = point_cache();
        std::lock_guard<std::mutex> lk(c.mu);
        c.max_bytes = max_bytes;
        if (max_bytes == 0) {
            drop.swap(c.entries);
            c.bytes = 0;
            c.hits = c.misses = 0;
        }
        while (c.bytes > c.max_bytes && !c.entries.empty()) {  // a lower limit
            size_t oldest = 0;
            for (size_t i = 1; i < c.entries.size(); ++i)
                if (c.entries[i]->last_use < c.entries[oldest]->last_use) oldest = i;
            c.bytes -= (int64_t)c.entries[oldest]->bytes;
            drop.push_back(c.entries[oldest]);
            c.entries.erase(c.entries.begin() + (long)oldest);
        }
    }
    return GIRG_OK;  // the dropped entries are freed here, outside the lock
}

int girg_point_cache_stats(int64_t* entries, int64_t* bytes, int64_t* hits, int64_t* misses) {
    PointCache& c = point_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (entries) *entries = (int64_t)c.entries.size();
    if (bytes) *bytes = c.bytes;
    if (hits) *hits = c.hits;
    if (misses) *misses = c.misses;
    return GIRG_OK;
}

int girg_scratch_pool_trim(int64_t keep_bytes) {
    if (keep_bytes < 0) return GIRG_E_PARAM;
    return guarded([&] {
        CK(cudaMemPoolTrimTo(library_pool(), (size_t)keep_bytes));
        return GIRG_OK;
    });
}

int girg_last_stats(int64_t* out, int32_t len) {
    const int k = len < kNumStats ? len : kNumStats;
    for (int q = 0; q < k; ++q) out[q] = g_stats[q];
    return k;
}

int girg_last_phase_ms(float* out, int32_t len) {
    const int k = len < 10 ? len : 10;
    for (int q = 0; q < k; ++q) out[q] = g_ms[q];
    return k;
}

int girg_points(int64_t n, int32_t d, double beta, double w_min, uint64_t seed, double* d_w,
                uint32_t* d_X, void* stream) {
    if (n < 1 || d < 1 || d > kMaxDim || !(beta > 2.0) || !(w_min > 0.0)) return GIRG_E_PARAM;
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        launch_girg_points(n, d, beta, w_min, seed, d_w, d_X, st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        return GIRG_OK;
    });
}

int hrg_points(int64_t n, double alpha, double R, uint64_t seed, double* d_r, uint32_t* d_X,
               void* stream) {
    if (n < 1 || !(alpha > 0.5) || !(R > 0.0)) return GIRG_E_PARAM;
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        launch_hrg_points(n, alpha, R, seed, d_r, nullptr, d_X, st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        return GIRG_OK;
    });
}

int hrg_girg_points(int64_t n, double alpha, double R, uint64_t seed, double* d_w, uint32_t* d_X,
                    void* stream) {
    if (n < 1 || !(alpha > 0.5) || !(R > 0.0) || !d_w || !d_X) return GIRG_E_PARAM;
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        Scratch S(st);
        double* r = S.get<double>(n);
        launch_hrg_points(n, alpha, R, seed, r, d_w, d_X, st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        return GIRG_OK;
    });
}

int girg_generate(const girg_params* params, void* d_edges, int64_t capacity_edges,
                  int64_t* num_edges, double* c_used, void* stream) {
    const int chk = check_girg(params);
    if (chk != GIRG_OK) return chk;
    if (!num_edges || capacity_edges < 0) return GIRG_E_PARAM;
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        d_edges = device_view(d_edges);
        Scratch S(st, scratch_reserve(*params));
        Timer tm(st);
        g_launches = 0;
        tm.mark();
        Problem P;
        P.model = 0;
        P.n = params->n;
        P.d = params->d;
        P.T = params->T;
        P.w_min = params->w_min;
        P.seed = params->seed;
        P.precision = params->precision;
        P.edge_bytes = params->edge_bytes;
        P.level_cap = params->level_cap;
        const bool caching = cache_on();
        CacheKey key{};
        if (caching) {
            int dev = 0;
            CK(cudaGetDevice(&dev));
            key = CacheKey{P.n, P.d, P.level_cap, dev, params->beta, P.w_min, P.T,
                           params->c > 0.0 ? params->c : 0.0,
                           params->c > 0.0 ? 0.0 : params->avg_deg, P.seed};
            if (std::shared_ptr<CacheEntry> e = point_cache().find(key)) {
                // a kept layout: no points, reductions, scale search or sort
                tm.mark();
                tm.mark();
                tm.mark();
                P.K = e->K;
                P.W = e->W;
                g_last_K = P.K;
                if (c_used) *c_used = e->c_used;
                run_sampler(P, e->Lo, S, st, tm, d_edges, capacity_edges, num_edges);
                finish_timing(tm);
                return P.edge_bytes != 0 && *num_edges > capacity_edges ? GIRG_E_CAPACITY : GIRG_OK;
            }
        }
        double* w = S.get<double>(P.n);
        uint32_t* X = S.get<uint32_t>((size_t)P.d * P.n);
        launch_girg_points(P.n, P.d, params->beta, P.w_min, P.seed, w, X, st);
        P.w = w;
        P.X = X;
        const bool solve = !(params->c > 0.0);
        const int E0 = exponent_of_ulp(P.w_min);
        Reduce* red = new_reduce(S, st);
        double* part_s2 = solve ? S.get<double>(reduce_blocks(P.n)) : nullptr;
        SplitDev D{};
        SplitHost* h = nullptr;
        if (solve) {  // the weight split for the degree model, before the one readback
            D = split_buffers(P.n, S);
            h = pinned_split();
            const ThresholdJob job{P.d, P.T, params->avg_deg, D.thr};
            launch_reduce(P.n, w, nullptr, P.w_min, E0, part_s2, red, st, &job);
            queue_split(P, D, h, st);
        } else {
            launch_reduce(P.n, w, nullptr, P.w_min, E0, nullptr, red, st);
        }
        tm.mark();
        auto h0 = std::chrono::steady_clock::now();
        read_reduce(P, red, st);
        g_ms[7] = (float)host_ms_since(h0);
        if (P.red.range_error) return GIRG_E_RANGE;
        P.W = round128(P.red.sum_hi, P.red.sum_lo, E0);
        h0 = std::chrono::steady_clock::now();
        P.K = solve ? solve_K(P, params->avg_deg, D, h, S, st) : girg_K_of_c(params->c, P.d, P.T);
        g_ms[8] = (float)host_ms_since(h0);
        g_last_K = P.K;
        const double cu = solve ? c_of_K(P.K, P.d, P.T) : params->c;
        if (c_used) *c_used = cu;
        if (caching) {  // build the layout into buffers the cache keeps
            auto e = std::make_shared<CacheEntry>();
            e->key = key;
            e->K = P.K;
            e->W = P.W;
            e->c_used = cu;
            Scratch A(st);  // frees what it holds if the build throws
            build_layout(P, A, S, st, tm, e->Lo, nullptr);
            e->bytes = A.bytes;
            e->bufs = A.release();
            run_sampler(P, e->Lo, S, st, tm, d_edges, capacity_edges, num_edges);  // syncs st
            finish_timing(tm);
            point_cache().insert(e);
            return P.edge_bytes != 0 && *num_edges > capacity_edges ? GIRG_E_CAPACITY : GIRG_OK;
        }
        Layout Lo;
        build_layout(P, S, S, st, tm, Lo, nullptr);
        run_sampler(P, Lo, S, st, tm, d_edges, capacity_edges, num_edges);
        finish_timing(tm);
        return P.edge_bytes != 0 && *num_edges > capacity_edges ? GIRG_E_CAPACITY : GIRG_OK;
    });
}

int girg_expected_avg_degree(const girg_params* params, double* avg_deg, void* stream) {
    if (!params || !avg_deg || !(params->c > 0.0)) return GIRG_E_PARAM;
    girg_params q = *params;
    const int chk = check_girg(&q);
    if (chk != GIRG_OK) return chk;
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        Scratch S(st);
        Problem P;
        P.n = q.n;
        P.d = q.d;
        P.T = q.T;
        P.w_min = q.w_min;
        double* w = S.get<double>(P.n);
        uint32_t* X = S.get<uint32_t>((size_t)P.d * P.n);
        launch_girg_points(P.n, P.d, q.beta, P.w_min, q.seed, w, X, st);
        P.w = w;
        const int E0 = exponent_of_ulp(P.w_min);
        Reduce* red = new_reduce(S, st);
        launch_reduce(P.n, w, nullptr, P.w_min, E0, nullptr, red, st);
        read_reduce(P, red, st);
        if (P.red.range_error) return GIRG_E_RANGE;
        P.W = round128(P.red.sum_hi, P.red.sum_lo, E0);
        double wmax = 0.0;
        for (int i = 0; i < kMaxLayers; ++i)
            if (P.red.cnt[i]) wmax = std::max(wmax, bits_to_double(P.red.wmax[i]));
        const double K = girg_K_of_c(q.c, P.d, P.T);
        // split below the weight at which E_R pairs can begin
        const double thr = 0.5 * P.W / (std::ldexp(K, P.d) * wmax);
        SplitDev D = split_buffers(P.n, S);
        SplitHost* h = pinned_split();
        CK(cudaMemcpyAsync(D.thr, &thr, sizeof(double), cudaMemcpyHostToDevice, st));
        queue_split(P, D, h, st);
        CK(cudaStreamSynchronize(st));
        DegreeModel M(P.n, P.d, P.T, P.W);
        take_split(P, M, D, h, S, st);
        *avg_deg = M.f(K);
        return GIRG_OK;
    });
}

static int from_points_impl(int64_t n, int32_t d, const uint32_t* d_X, const double* d_w, double T,
                            double c, uint64_t seed, int32_t precision, int32_t level_cap,
                            int32_t edge_bytes, void* d_edges, int64_t capacity_edges,
                            int64_t* num_edges, int64_t* order_out, void* stream) {
    if (n < 2 || n >= (1ll << 31) || d < 1 || d > kMaxDim || !(T >= 0.0 && T < 1.0) || !(c > 0.0))
        return GIRG_E_PARAM;
    if ((edge_bytes != 0 && edge_bytes != 4 && edge_bytes != 8) || (precision != 0 && precision != 1) ||
        level_cap < 0)
        return GIRG_E_PARAM;
    if (!order_out && (!num_edges || capacity_edges < 0)) return GIRG_E_PARAM;
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        girg_params est{};
        est.n = n;
        est.d = d;
        est.T = T;
        Scratch S(st, order_out ? 0 : scratch_reserve(est));
        Timer tm(st);
        g_launches = 0;
        tm.mark();
        Problem P;
        P.n = n;
        P.d = d;
        P.T = T;
        P.K = girg_K_of_c(c, d, T);
        g_last_K = P.K;
        P.seed = seed;
        P.precision = precision;
        P.edge_bytes = edge_bytes;
        P.level_cap = level_cap;
        P.X = d_X;
        P.w = d_w;
        unsigned long long* mn = S.get<unsigned long long>(1);
        CK(cudaMemsetAsync(mn, 0xff, sizeof(unsigned long long), st));
        launch_min_weight(n, d_w, mn, st);
        unsigned long long mb = 0;
        CK(cudaMemcpyAsync(&mb, mn, sizeof(mb), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        P.w_min = bits_to_double(mb);
        if (!(P.w_min > 0.0)) return GIRG_E_PARAM;
        const int E0 = exponent_of_ulp(P.w_min);
        Reduce* red = new_reduce(S, st);
        launch_reduce(n, d_w, nullptr, P.w_min, E0, nullptr, red, st);
        tm.mark();
        read_reduce(P, red, st);
        if (P.red.range_error) return GIRG_E_RANGE;
        P.W = round128(P.red.sum_hi, P.red.sum_lo, E0);
        int64_t dummy = 0;
        Layout Lo;
        build_layout(P, S, S, st, tm, Lo, order_out);
        if (order_out) return GIRG_OK;
        run_sampler(P, Lo, S, st, tm, d_edges, capacity_edges, num_edges ? num_edges : &dummy);
        finish_timing(tm);
        return edge_bytes != 0 && *num_edges > capacity_edges ? GIRG_E_CAPACITY : GIRG_OK;
    });
}

int girg_generate_from_points(int64_t n, int32_t d, const uint32_t* d_X, const double* d_w,
                              double T, double c, uint64_t seed, int32_t precision,
                              int32_t level_cap, int32_t edge_bytes, void* d_edges,
                              int64_t capacity_edges, int64_t* num_edges, void* stream) {
    return from_points_impl(n, d, d_X, d_w, T, c, seed, precision, level_cap, edge_bytes, d_edges,
                            capacity_edges, num_edges, nullptr, stream);
}

int girg_sorted_order(int64_t n, int32_t d, const uint32_t* d_X, const double* d_w, double T,
                      double c, int32_t level_cap, int64_t* d_order, void* stream) {
    if (!d_order) return GIRG_E_PARAM;
    return from_points_impl(n, d, d_X, d_w, T, c, 0, 0, level_cap, 4, nullptr, 0, nullptr,
                            d_order, stream);
}

static bool hrg_shape_ok(int64_t n, double alpha, double T) {
    return n >= 2 && n < (1ll << 31) && alpha > 0.5 && alpha < 1e6 && T >= 0.0 && T < 1.0;
}

int hrg_expected_avg_degree(int64_t n, double alpha, double T, double R, double* avg_deg) {
    if (!avg_deg || !hrg_shape_ok(n, alpha, T) || !(R > 0.0 && R <= 350.0)) return GIRG_E_PARAM;
    *avg_deg = hrg_expected_degree(n, alpha, T, R);
    return GIRG_OK;
}

int hrg_solve_radius(int64_t n, double alpha, double T, double avg_deg, double* R) {
    if (!R || !hrg_shape_ok(n, alpha, T) || !(avg_deg > 0.0 && avg_deg < (double)(n - 1)))
        return GIRG_E_PARAM;
    const double r = hrg_radius_for_degree(n, alpha, T, avg_deg);
    if (!(r > 0.0 && r <= 350.0)) return GIRG_E_PARAM;
    *R = r;
    return GIRG_OK;
}

// The radius for a target degree at T > 0 with the distance CDF of every node of the
// logistic t rule evaluated on the device (one launch and one readback per step of
// the search); the search itself and the sums over the nodes stay on the host.
double hrg_radius_on_device(const hrg_params& q, Scratch& S, cudaStream_t st) {
    HrgYRule Y;
    Y.n = kHrgYNodes;
    static_assert(kHrgYNodes <= kHrgYMax, "y rule fits");
    hrg_unit_y_rule(Y.c, Y.w);
    constexpr int kMaxNodes = 512;  // the t rule has at most 12 intervals of 20 nodes
    double* d_ts = S.get<double>(kMaxNodes);
    double* d_g = S.get<double>(4 * kMaxNodes);
    std::vector<double> ts, ws, g;
    auto E = [&](double R) {
        double tail = 0.0;
        hrg_t_rule(R, q.T, ts, ws, &tail);
        const int nt = (int)ts.size();
        if (nt > kMaxNodes) throw Status{GIRG_E_INTERNAL};
        g.assign(4 * (size_t)nt, 0.0);
        CK(cudaMemcpyAsync(d_ts, ts.data(), nt * sizeof(double), cudaMemcpyHostToDevice, st));
        launch_hrg_dist_cdf(q.alpha, R, Y, d_ts, nt, d_g, st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(g.data(), d_g, 4 * nt * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double p = 0.0;
        for (int i = 0; i < nt; ++i) p += ws[i] * (((g[4 * i] + g[4 * i + 1]) + g[4 * i + 2]) + g[4 * i + 3]);
        p += tail;
        return (double)(q.n - 1) * p;
    };
    return hrg_radius_for_degree(q.n, q.alpha, q.T, q.avg_deg, E);
}

int hrg_generate(const hrg_params* params, void* d_edges, int64_t capacity_edges,
                 int64_t* num_edges, double* R_used, void* stream) {
    if (!params || !num_edges || capacity_edges < 0) return GIRG_E_PARAM;
    hrg_params q = *params;
    if (!hrg_shape_ok(q.n, q.alpha, q.T) || !(q.R <= 350.0)) return GIRG_E_PARAM;
    if ((q.edge_bytes != 0 && q.edge_bytes != 4 && q.edge_bytes != 8) ||
        (q.precision != 0 && q.precision != 1) ||
        q.level_cap < 0)
        return GIRG_E_PARAM;
    const bool solve = !(q.R > 0.0);
    if (solve && !(q.avg_deg > 0.0 && q.avg_deg < (double)(q.n - 1))) return GIRG_E_PARAM;
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        girg_params est{};
        est.n = q.n;
        est.d = 1;
        est.T = q.T;
        Scratch S(st, scratch_reserve(est));
        for (int k = 7; k <= 9; ++k) g_ms[k] = 0.0f;
        if (solve) {  // the radius for the target degree (host search)
            const auto h0 = std::chrono::steady_clock::now();
            q.R = q.T > 0.0 ? hrg_radius_on_device(q, S, st)
                            : hrg_radius_for_degree(q.n, q.alpha, q.T, q.avg_deg);
            g_ms[8] = (float)host_ms_since(h0);
            if (!(q.R > 0.0 && q.R <= 350.0)) return GIRG_E_PARAM;
        }
        if (R_used) *R_used = q.R;
        Timer tm(st);
        g_launches = 0;
        tm.mark();
        Problem P;
        P.model = 1;
        P.n = q.n;
        P.d = 1;
        P.T = q.T;
        P.R = q.R;
        P.alpha = q.alpha;
        P.w_min = 1.0;
        P.seed = q.seed;
        P.precision = q.precision;
        P.edge_bytes = q.edge_bytes;
        P.level_cap = q.level_cap;
        double* r = S.get<double>(P.n);
        double* w = S.get<double>(P.n);
        uint32_t* X = S.get<uint32_t>(P.n);
        launch_hrg_points(P.n, q.alpha, q.R, q.seed, r, w, X, st);
        P.r = r;
        P.w = w;
        P.X = X;
        Reduce* red = new_reduce(S, st);
        launch_reduce(P.n, w, r, 1.0, exponent_of_ulp(1.0), nullptr, red, st);
        tm.mark();
        const auto h1 = std::chrono::steady_clock::now();
        read_reduce(P, red, st);  // the HRG needs no weight sum: a range error is harmless
        g_ms[7] = (float)host_ms_since(h1);
        P.W = 1.0;
        Layout Lo;
        build_layout(P, S, S, st, tm, Lo, nullptr);
        run_sampler(P, Lo, S, st, tm, d_edges, capacity_edges, num_edges);
        finish_timing(tm);
        return P.edge_bytes != 0 && *num_edges > capacity_edges ? GIRG_E_CAPACITY : GIRG_OK;
    });
}

int girg_allpairs(int64_t n, int32_t d, const uint32_t* d_X, const double* d_w, double W,
                  double T, double c, uint64_t seed, int32_t precision, int32_t edge_bytes,
                  void* d_edges, int64_t capacity_edges, int64_t* num_edges, void* stream) {
    if (n < 2 || n >= (1ll << 31) || d < 1 || d > kMaxDim || !(T >= 0.0 && T < 1.0) || !(c > 0.0) ||
        !(W > 0.0) || !num_edges || capacity_edges < 0)
        return GIRG_E_PARAM;
    if ((edge_bytes != 4 && edge_bytes != 8) || (precision != 0 && precision != 1)) return GIRG_E_PARAM;
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        d_edges = device_view(d_edges);
        Scratch S(st);
        float* sv = S.get<float>(n);
        const bool tzero = T == 0.0;
        const double K = girg_K_of_c(c, d, T);
        const float gamma = (float)(std::log2(K) / (2.0 * d));
        launch_scale(n, d_w, 0.5 * std::log2(W), gamma, (float)(1.0 / d), sv, st);
        unsigned long long* stats = S.get<unsigned long long>(kNumStats + 2);
        CK(cudaMemsetAsync(stats, 0, (kNumStats + 2) * sizeof(unsigned long long), st));
        DevCfg cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.n = (int32_t)n;
        cfg.d = d;
        cfg.precision = precision;
        cfg.tzero = tzero ? 1 : 0;
        const double invT = T > 0.0 ? 1.0 / T : 0.0;
        cfg.invT = invT;
        cfg.m_int = (T > 0.0 && invT == std::floor(invT) && invT <= 64.0) ? (int)invT : 0;
        cfg.seed_lo = (uint32_t)seed;
        cfg.seed_hi = (uint32_t)(seed >> 32);
        cfg.W = W;
        cfg.K = K;
        cfg.T = T;
        cfg.dT = T > 0.0 ? (float)(d / T) : 0.0f;
        cfg.bandG = cfg.dT * 0x1p-14f + 0x1p-15f;
        cfg.band_ratio = 0x1p-16f;
        cfg.edges = d_edges;
        cfg.edge_bytes = edge_bytes;
        cfg.cap = capacity_edges;
        cfg.edge_count = stats + kNumStats;
        cfg.stats = stats;
        launch_allpairs(cfg, d_X, d_w, sv, st);
        unsigned long long m = 0;
        CK(cudaMemcpyAsync(&m, stats + kNumStats, sizeof(m), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        *num_edges = (int64_t)m;
        return *num_edges > capacity_edges ? GIRG_E_CAPACITY : GIRG_OK;
    });
}

}  // extern "C"
