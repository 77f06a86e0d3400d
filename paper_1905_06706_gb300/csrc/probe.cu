// girg_issue_probe: the warp-instruction issue rate this GPU reaches, measured.
//
// The pair-test and jump kernels are bound by instruction issue, not by memory
// bandwidth (each pair is a Philox draw and a few dozen integer and FP32 operations
// on data that sits in L1/L2).  The denominator of their roofline is therefore the
// rate at which the SMs issue warp instructions of the kinds those kernels execute.
// This probe measures it: every resident warp runs long runs of one instruction kind
// (integer logic, integer multiply-add, FP32 fused multiply-add) over eight
// independent register chains whose operands are runtime values, so that the issue
// slots, not dependences or memory, limit the rate.  The grid fills every SM (two
// 1024-thread blocks per SM).  The paper has no counterpart: its experiments time a
// CPU.
#include <cuda_runtime.h>

#include <cstdint>

#include "girg_gb300.h"
#include "kernels.h"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeBlocksPerSm = 2;
constexpr int kOpsPerIter = 128;  // four asm blocks of 32 operations

// Written only when the chains reach an impossible value: keeps the chains live.
__device__ unsigned int g_probe_sink;

#define GG_LOP3_8                                                                       \
    "lop3.b32 %0, %0, %1, %8, 0x96;\n\tlop3.b32 %1, %1, %2, %8, 0x96;\n\t"              \
    "lop3.b32 %2, %2, %3, %8, 0x96;\n\tlop3.b32 %3, %3, %4, %8, 0x96;\n\t"              \
    "lop3.b32 %4, %4, %5, %8, 0x96;\n\tlop3.b32 %5, %5, %6, %8, 0x96;\n\t"              \
    "lop3.b32 %6, %6, %7, %8, 0x96;\n\tlop3.b32 %7, %7, %0, %8, 0x96;\n\t"
#define GG_IMAD_8                                                                       \
    "mad.lo.u32 %0, %0, %1, %8;\n\tmad.lo.u32 %1, %1, %2, %8;\n\t"                      \
    "mad.lo.u32 %2, %2, %3, %8;\n\tmad.lo.u32 %3, %3, %4, %8;\n\t"                      \
    "mad.lo.u32 %4, %4, %5, %8;\n\tmad.lo.u32 %5, %5, %6, %8;\n\t"                      \
    "mad.lo.u32 %6, %6, %7, %8;\n\tmad.lo.u32 %7, %7, %0, %8;\n\t"
#define GG_FFMA_8                                                                       \
    "fma.rn.f32 %0, %0, %1, %8;\n\tfma.rn.f32 %1, %1, %2, %8;\n\t"                      \
    "fma.rn.f32 %2, %2, %3, %8;\n\tfma.rn.f32 %3, %3, %4, %8;\n\t"                      \
    "fma.rn.f32 %4, %4, %5, %8;\n\tfma.rn.f32 %5, %5, %6, %8;\n\t"                      \
    "fma.rn.f32 %6, %6, %7, %8;\n\tfma.rn.f32 %7, %7, %0, %8;\n\t"

// 32 operations of one kind on the eight chains a[0..7] with the runtime operand k.
template <int KIND>
__device__ __forceinline__ void ops32(unsigned int (&a)[8], unsigned int k) {
    static_assert(KIND == 0 || KIND == 1, "integer kinds");
    if constexpr (KIND == 0) {
        asm volatile(GG_LOP3_8 GG_LOP3_8 GG_LOP3_8 GG_LOP3_8
                     : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]),
                       "+r"(a[5]), "+r"(a[6]), "+r"(a[7])
                     : "r"(k));
    } else if constexpr (KIND == 1) {
        asm volatile(GG_IMAD_8 GG_IMAD_8 GG_IMAD_8 GG_IMAD_8
                     : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]),
                       "+r"(a[5]), "+r"(a[6]), "+r"(a[7])
                     : "r"(k));
    }
}

__device__ __forceinline__ void ops32(float (&a)[8], float k) {
    asm volatile(GG_FFMA_8 GG_FFMA_8 GG_FFMA_8 GG_FFMA_8
                 : "+f"(a[0]), "+f"(a[1]), "+f"(a[2]), "+f"(a[3]), "+f"(a[4]), "+f"(a[5]),
                   "+f"(a[6]), "+f"(a[7])
                 : "f"(k));
}

#undef GG_LOP3_8
#undef GG_IMAD_8
#undef GG_FFMA_8

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
    k_issue_probe(int64_t iters, unsigned int seed, unsigned int never) {
    const unsigned int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int x = 0;
    if constexpr (KIND == 2) {
        // chains start in [1/2, 1); a * b + 2^-24 with a, b in (0, 1) stays in
        // [2^-24, 1): finite and normal throughout
        float a[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = 0.5f + (float)((t * 8u + i) & 1023u) * 0x1p-11f;
        const float k = 0x1p-24f;
        for (int64_t it = 0; it < iters; ++it) {
            ops32(a, k);
            ops32(a, k);
            ops32(a, k);
            ops32(a, k);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) x ^= __float_as_uint(a[i]);
    } else {
        unsigned int a[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = (t * 8u + i) ^ seed;
        for (int64_t it = 0; it < iters; ++it) {
            ops32<KIND>(a, seed);
            ops32<KIND>(a, seed);
            ops32<KIND>(a, seed);
            ops32<KIND>(a, seed);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) x ^= a[i];
    }
    if (x == never) g_probe_sink = x;
}

}  // namespace

extern "C" int girg_issue_probe(int32_t kind, int64_t iters, void* stream, float* ms,
                                int64_t* warp_instructions) {
    if (kind < 0 || kind > 2 || iters < 1 || iters > (int64_t(1) << 24) || !ms ||
        !warp_instructions)
        return GIRG_E_PARAM;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = gg::device_sms() * kProbeBlocksPerSm;
    if (blocks <= 0) return GIRG_E_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return GIRG_E_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GIRG_E_CUDA;
    }
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        const unsigned int seed = 0x9e3779b9u, never = 0x0badf00du;
        if (kind == 0)
            k_issue_probe<0><<<blocks, kProbeThreads, 0, s>>>(iters, seed, never);
        else if (kind == 1)
            k_issue_probe<1><<<blocks, kProbeThreads, 0, s>>>(iters, seed, never);
        else
            k_issue_probe<2><<<blocks, kProbeThreads, 0, s>>>(iters, seed, never);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return GIRG_E_CUDA;
    *warp_instructions = (int64_t)blocks * (kProbeThreads / 32) * iters * kOpsPerIter;
    return GIRG_OK;
}
