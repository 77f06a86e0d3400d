// girg_allpairs_noalloc: the all-pairs generator with no device allocation.
//
// Some callers cannot allocate device memory: a plug-in running inside a host
// application that owns the whole device memory pool and forbids allocations of
// its own, or a latency-critical loop where cudaMalloc could block on the device
// or fail under memory pressure.  This variant of girg_allpairs therefore keeps
// its scratch (the per-vertex single-precision scale and the edge/statistics
// counters) in one fixed file-scope device array instead of allocating it.  The
// paper has no counterpart of this entry point.
//
// The array lives for as long as the library stays loaded, on every GPU that
// loads it.  Every call uses the same array, so calls whose device work overlaps
// (on different streams or host threads) race on it and must be serialised by
// the caller.
#include <cmath>
#include <cstring>
#include <mutex>

#include "girg_gb300.h"
#include "internal.cuh"
#include "kernels.h"

using namespace gg;

namespace {

constexpr int64_t kMaxN = GIRG_NOALLOC_MAX_N;
constexpr int kCounterWords = kNumStats + 2;  // statistics, edge count, spare
constexpr size_t kScaleBytes = ((size_t)kMaxN * sizeof(float) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kScaleBytes + kCounterWords * sizeof(unsigned long long);

// The fixed scratch: [0, kScaleBytes) per-vertex scale, then the counters.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in, so the
// kernels receive this address instead.
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// A caller pointer as the kernels see it: device (or managed) memory as given,
// page-locked host memory mapped into the device through its device pointer.
// Anything else -- pageable host memory, a pointer CUDA does not know -- returns
// GIRG_E_PARAM before any device work, so a bad pointer becomes a status instead of
// a memory fault on the GPU.
int device_view(const void* p, void** out) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error state of a failed lookup
        return GIRG_E_PARAM;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        *out = const_cast<void*>(p);
        return GIRG_OK;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *out = a.devicePointer;
        return GIRG_OK;
    }
    return GIRG_E_PARAM;
}

}  // namespace

extern "C" int girg_allpairs_noalloc(int64_t n, int32_t d, const uint32_t* d_X, const double* d_w,
                                     double W, double T, double c, uint64_t seed,
                                     int32_t precision, int32_t edge_bytes, void* d_edges,
                                     int64_t capacity_edges, int64_t* num_edges, void* stream) {
    if (n < 2 || n > kMaxN || d < 1 || d > kMaxDim || !(T >= 0.0 && T < 1.0) || !(c > 0.0) ||
        !(W > 0.0) || !num_edges || capacity_edges < 0)
        return GIRG_E_PARAM;
    if ((edge_bytes != 4 && edge_bytes != 8) || (precision != 0 && precision != 1))
        return GIRG_E_PARAM;
    void *edges = nullptr, *X = nullptr, *w = nullptr;
    if (device_view(d_edges, &edges) != GIRG_OK || device_view(d_X, &X) != GIRG_OK ||
        device_view(d_w, &w) != GIRG_OK)
        return GIRG_E_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return GIRG_E_CUDA;
    float* sv = reinterpret_cast<float*>(base);
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(base + kScaleBytes);
    // the counters must start at zero; the scale array is fully rewritten
    if (cudaMemsetAsync(counters, 0, kCounterWords * sizeof(unsigned long long), st) != cudaSuccess)
        return GIRG_E_CUDA;
    const bool tzero = T == 0.0;
    const double K = girg_K_of_c(c, d, T);
    const float gamma = (float)(std::log2(K) / (2.0 * d));
    launch_scale(n, static_cast<const double*>(w), 0.5 * std::log2(W), gamma, (float)(1.0 / d), sv,
                 st);
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
    cfg.edges = edges;
    cfg.edge_bytes = edge_bytes;
    cfg.cap = capacity_edges;
    cfg.stats = counters;
    cfg.edge_count = counters + kNumStats;
    if (!det_tables_pairs()) return GIRG_E_CUDA;
    launch_allpairs(cfg, static_cast<const uint32_t*>(X), static_cast<const double*>(w), sv, st);
    unsigned long long m = 0;
    if (cudaMemcpyAsync(&m, counters + kNumStats, sizeof(m), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return GIRG_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return GIRG_E_CUDA;
    *num_edges = (int64_t)m;
    return *num_edges > capacity_edges ? GIRG_E_CAPACITY : GIRG_OK;
}
