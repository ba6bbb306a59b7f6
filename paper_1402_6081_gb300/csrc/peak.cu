// Measured arithmetic peak of the current GPU: the denominator of the FP32
// and FP64 rooflines of the products and transforms (no counterpart in the
// paper).  Every SM runs as many CTAs as fit, each thread a set of independent
// chains of fused multiply-adds of one kind, written as inline PTX so the
// compiler neither merges nor drops them; CUDA events time each launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "lgf_internal.h"

namespace lgf {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 16;   // independent accumulators per thread

// kind 0: fma.rn.f64, 1: fma.rn.f32, 2: fma.rn.f32x2 (two lanes per instruction)
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, double* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (KIND == 0) {
        double acc[kChains];
        const double m = 0.999999999, a = 1e-9 * (t & 7);
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = 1.0 + c * 1e-3;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(acc[c]) : "d"(m), "d"(a));
        }
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += acc[c];
        if (s == -1.0) out[t] = s;   // never true: keeps the chains live
    } else if constexpr (KIND == 1) {
        float acc[kChains];
        const float m = 0.9999999f, a = 1e-7f * float(t & 7);
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = 1.0f + c * 1e-3f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(acc[c]) : "f"(m), "f"(a));
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += acc[c];
        if (s == -1.f) out[t] = s;
    } else {
        uint64_t acc[kChains], m, a;
        const float mf = 0.9999999f, af = 1e-7f * float(t & 7);
        asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(mf));
        asm("mov.b64 %0, {%1, %1};" : "=l"(a) : "f"(af));
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const float v = 1.0f + c * 1e-3f;
            asm("mov.b64 %0, {%1, %1};" : "=l"(acc[c]) : "f"(v));
        }
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[c]) : "l"(m), "l"(a));
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[c]));
            s += lo + hi;
        }
        if (s == -1.f) out[t] = s;
    }
}

template <int KIND>
cudaError_t launch_peak(int grid, int iters, double* out, cudaStream_t st) {
    k_fma_peak<KIND><<<grid, kPeakThreads, 0, st>>>(iters, out);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t resident_ctas(int* n) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_fma_peak<KIND>, kPeakThreads, 0);
}

}  // namespace
}  // namespace lgf

extern "C" lgf_status lgf_measure_fma_peak(int32_t kind, int32_t reps, double* flops_per_s, double* ms) {
    using namespace lgf;
    if (kind < 0 || kind > 2 || reps < 1 || reps > 100 || !flops_per_s || !ms)
        return fail(LGF_ERR_INVALID_ARG, "lgf_measure_fma_peak: need kind 0..2, 1 <= reps <= 100 and outputs");
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = kind == 0 ? resident_ctas<0>(&per_sm) : kind == 1 ? resident_ctas<1>(&per_sm)
                                                                                : resident_ctas<2>(&per_sm);
    if (e != cudaSuccess) return fail(LGF_ERR_CUDA, std::string("lgf_measure_fma_peak: ") + cudaGetErrorString(e));
    const int grid = n_sm * std::max(1, per_sm);
    // about 20-60 ms per launch at the GB300's rates
    const int iters = kind == 0 ? 4096 : kind == 1 ? 131072 : 65536;
    const double lanes = kind == 2 ? 2.0 : 1.0;
    double* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&out, sizeof(double) * size_t(grid) * kPeakThreads);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 0.f;
    for (int r = 0; e == cudaSuccess && r <= reps; ++r) {
        e = cudaEventRecord(a, 0);
        if (e == cudaSuccess)
            e = kind == 0 ? launch_peak<0>(grid, iters, out, 0) : kind == 1 ? launch_peak<1>(grid, iters, out, 0)
                                                                           : launch_peak<2>(grid, iters, out, 0);
        if (e == cudaSuccess) e = cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e == cudaSuccess && r > 0 && (best == 0.f || t < best)) best = t;   // r = 0 is the warm-up
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return fail(LGF_ERR_CUDA, std::string("lgf_measure_fma_peak: ") + cudaGetErrorString(e));
    const double fmas = double(grid) * kPeakThreads * double(iters) * kChains * lanes;
    *ms = best;
    *flops_per_s = 2.0 * fmas / (double(best) * 1e-3);
    return ok();
}
