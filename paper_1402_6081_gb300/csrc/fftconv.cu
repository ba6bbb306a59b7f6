// FFT convolution of isolated blocks in one kernel (lgf_conv_blocks): every
// block is its own single-block domain, the special case where the FLGF method
// reduces to one zero-padded FFT convolution (Sec. 4.2, "FFT Conv."; Eqs.
// alg_upfft, alg_mult with the block's own kernel spectrum only, alg_dwfft).
//
// With one block per domain the three steps of Sec. 3.1 are local to the
// block, so one CTA takes a block through all of them with its spectrum in
// shared memory: the forward x and y passes fill the partially transformed
// cube (z < n planes of S x NX), the z pass transforms each (kx, ky) line,
// multiplies it by the kernel spectrum, transforms it back and keeps its first
// n values in place, and the inverse y and x passes end in the output block.
// The spectrum never leaves the SM; the kernel spectrum (139 KB at n_b = 16,
// FP32) is read by every block and stays in L2.  The arithmetic is that of the
// three-launch path (the per-block transforms of kernels_impl.cuh, the product
// as cmac(0, f, k)), in the same order.
//
// State per device: this unit's twiddle tables and the kernel spectrum of each
// (n_b, precision) used, made on the first call that needs them (synchronous
// uploads: make the first call before any stream capture).
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels_impl.cuh"

namespace lgf {
namespace conv {

using dev::cx;
using dev::czero;

template <typename T, int S, int N>
__global__ void __launch_bounds__(dev::fft_threads<T, S, N>(), dev::fft_min_blocks<T, S, N>())
    k_conv(const T* __restrict__ f, T* __restrict__ u, const cx<T>* __restrict__ kh, int n_items) {
    constexpr int NX = S / 2 + 1, NXP = NX | 1, PP = (S * NXP) | 1;
    constexpr int K = dev::fft_items_per_cta<T, S, N>();
    constexpr size_t ITEM = sizeof(cx<T>) * size_t(N) * PP;
    constexpr int64_t B3 = int64_t(N) * N * N;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int first = blockIdx.x * K;
    const int nk = min(K, n_items - first);
    auto Bof = [&](int b) { return reinterpret_cast<cx<T>*>(smem_raw + b * ITEM); };

    // forward x pass: rows l0 and l0 + NP of the (y, z) plane as one complex line
    constexpr int NL = N * N, NP = (NL + 1) / 2;
    for (int p = threadIdx.x; p < nk * NP; p += blockDim.x) {
        const int b = p / NP, l0 = p % NP, l1 = l0 + NP;
        const bool has1 = l1 < NL;
        const T* in = f + int64_t(first + b) * B3;
        cx<T> z[S];
#pragma unroll
        for (int x = 0; x < S; ++x)
            z[x] = x < N ? cx<T>{__ldg(in + l0 * N + x), has1 ? __ldg(in + l1 * N + x) : T(0)} : czero<T>();
        dev::fft<S, S, -1, N>(z);
        cx<T>* B = Bof(b);
        cx<T>* d0 = B + (l0 / N) * PP + (l0 % N) * NXP;
        cx<T>* d1 = B + (l1 / N) * PP + (l1 % N) * NXP;
#pragma unroll
        for (int k = 0; k < NX; ++k) {
            const cx<T> a = z[k], c = z[(S - k) % S];
            d0[k] = {T(0.5) * (a.x + c.x), T(0.5) * (a.y - c.y)};
            if (has1) d1[k] = {T(0.5) * (a.y + c.y), T(0.5) * (c.x - a.x)};
        }
    }
    __syncthreads();
    // forward y pass: lines (kx, z < N)
    for (int q = threadIdx.x; q < nk * NX * N; q += blockDim.x) {
        const int b = q / (NX * N), l = q % (NX * N);
        cx<T>* col = Bof(b) + (l / NX) * PP + l % NX;
        cx<T> v[S];
#pragma unroll
        for (int y = 0; y < S; ++y) v[y] = y < N ? col[y * NXP] : czero<T>();
        dev::fft<S, S, -1, N>(v);
#pragma unroll
        for (int y = 0; y < S; ++y) col[y * NXP] = v[y];
    }
    __syncthreads();
    // z pass: forward transform of the line, the product with the kernel
    // spectrum, the inverse transform; the first N values stay in place
    for (int q = threadIdx.x; q < nk * NX * S; q += blockDim.x) {
        const int b = q / (NX * S), l = q % (NX * S);
        cx<T>* col = Bof(b) + (l / NX) * NXP + l % NX;
        cx<T> v[S];
#pragma unroll
        for (int zz = 0; zz < S; ++zz) v[zz] = zz < N ? col[zz * PP] : czero<T>();
        dev::fft<S, S, -1, N>(v);
#pragma unroll
        for (int kz = 0; kz < S; ++kz) v[kz] = dev::cmac(czero<T>(), v[kz], dev::ldg_cx(kh + kz * S * NX + l));
        dev::fft<S, S, 1, S>(v);
#pragma unroll
        for (int zz = 0; zz < N; ++zz) col[zz * PP] = v[zz];
    }
    __syncthreads();
    // inverse y pass: lines (kx, z < N); keep y < N
    for (int q = threadIdx.x; q < nk * NX * N; q += blockDim.x) {
        const int b = q / (NX * N), l = q % (NX * N);
        cx<T>* col = Bof(b) + (l / NX) * PP + l % NX;
        cx<T> v[S];
#pragma unroll
        for (int y = 0; y < S; ++y) v[y] = col[y * NXP];
        dev::fft<S, S, 1, S>(v);
#pragma unroll
        for (int y = 0; y < N; ++y) col[y * NXP] = v[y];
    }
    __syncthreads();
    // inverse x pass: two Hermitian half-rows per complex inverse, the first N
    // samples of each to the output block
    for (int p = threadIdx.x; p < nk * NP; p += blockDim.x) {
        const int b = p / NP, l0 = p % NP, l1 = l0 + NP;
        const bool has1 = l1 < NL;
        const cx<T>* B = Bof(b);
        const cx<T>* ra = B + (l0 / N) * PP + (l0 % N) * NXP;
        const cx<T>* rb = B + (has1 ? (l1 / N) * PP + (l1 % N) * NXP : (l0 / N) * PP + (l0 % N) * NXP);
        cx<T> z[S];
#pragma unroll
        for (int k = 0; k < NX; ++k) {
            cx<T> A = ra[k], Bk = has1 ? rb[k] : czero<T>();
            if (k == 0 || 2 * k == S) {   // exactly real for a real signal
                A.y = T(0);
                Bk.y = T(0);
            }
            z[k] = {A.x - Bk.y, A.y + Bk.x};
            if (k > 0 && S - k >= NX) z[S - k] = {A.x + Bk.y, Bk.x - A.y};
        }
        dev::fft<S, S, 1, S>(z);
        T* out = u + int64_t(first + b) * B3;
#pragma unroll
        for (int x = 0; x < N; ++x) {
            out[l0 * N + x] = z[x].x;
            if (has1) out[l1 * N + x] = z[x].y;
        }
    }
}

template <typename T, int S, int N>
cudaError_t launch(const T* f, T* u, const cx<T>* kh, int64_t n, cudaStream_t st) {
    constexpr int K = dev::fft_items_per_cta<T, S, N>();
    constexpr int NX = S / 2 + 1, PP = (S * (NX | 1)) | 1;
    constexpr size_t smem = K * sizeof(cx<T>) * size_t(N) * PP;
    auto k = k_conv<T, S, N>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k<<<unsigned((n + K - 1) / K), dev::fft_threads<T, S, N>(), smem, st>>>(f, u, kh, int(n));
    return cudaGetLastError();
}

template <typename T>
cudaError_t upload_twiddles() {
    T c[dev::kTwTotal], s[dev::kTwTotal];
    for (int S : dev::kTwSizes) {
        const int o = dev::tw_offset(S);
        for (int j = 0; j < S; ++j) {
            const double a = 2.0 * M_PI * double(j) / double(S);
            c[o + j] = T(std::cos(a));
            s[o + j] = T(std::sin(a));
        }
    }
    if constexpr (sizeof(T) == 8) {
        cudaError_t e = cudaMemcpyToSymbol(dev::c_cos_d, c, sizeof(c));
        return e == cudaSuccess ? cudaMemcpyToSymbol(dev::c_sin_d, s, sizeof(s)) : e;
    } else {
        cudaError_t e = cudaMemcpyToSymbol(dev::c_cos_f, c, sizeof(c));
        return e == cudaSuccess ? cudaMemcpyToSymbol(dev::c_sin_f, s, sizeof(s)) : e;
    }
}

std::mutex g_mu;
std::map<int, bool> g_twiddles;                          // device -> uploaded
std::map<std::tuple<int, int, int>, void*> g_kernels;    // (device, n_b, precision) -> kernel spectrum

lgf_status cuda_fail_conv(cudaError_t e, const char* what) {
    cudaGetLastError();
    return fail(LGF_ERR_CUDA, std::string("lgf_conv_blocks: ") + what + ": " + cudaGetErrorString(e));
}

// The block's kernel spectrum (offset d = 0, level 0, 1/S^3 folded in), FP64
// on the host, rounded to the precision; made once per device.
lgf_status kernel_for(int device, int n_b, int prec, const void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    cudaError_t e;
    if (!g_twiddles[device]) {
        if ((e = upload_twiddles<float>()) != cudaSuccess) return cuda_fail_conv(e, "twiddle upload");
        if ((e = upload_twiddles<double>()) != cudaSuccess) return cuda_fail_conv(e, "twiddle upload");
        g_twiddles[device] = true;
    }
    auto key = std::make_tuple(device, n_b, prec);
    auto it = g_kernels.find(key);
    if (it != g_kernels.end()) {
        *out = it->second;
        return ok();
    }
    const int S = 2 * n_b;
    const int64_t NW = nw_of(S);
    auto tab = green_abs_table(1, n_b - 1);
    std::vector<std::complex<double>> kh(static_cast<size_t>(NW));
    const int d[3] = {0, 0, 0};
    kernel_spectrum(n_b, n_b, 1, S, d, tab->data(), n_b - 1, kh.data());
    const size_t elem = prec == LGF_FP64 ? sizeof(double) : sizeof(float);
    void* dev_ptr = nullptr;
    if ((e = cudaMalloc(&dev_ptr, 2 * elem * size_t(NW))) != cudaSuccess) {
        cudaGetLastError();
        return fail(LGF_ERR_OOM, "lgf_conv_blocks: kernel spectrum allocation");
    }
    if (prec == LGF_FP64) {
        e = cudaMemcpy(dev_ptr, kh.data(), 2 * elem * size_t(NW), cudaMemcpyHostToDevice);
    } else {
        std::vector<float> fl(2 * size_t(NW));
        for (size_t i = 0; i < size_t(NW); ++i) {
            fl[2 * i] = float(kh[i].real());
            fl[2 * i + 1] = float(kh[i].imag());
        }
        e = cudaMemcpy(dev_ptr, fl.data(), sizeof(float) * fl.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(dev_ptr);
        return cuda_fail_conv(e, "kernel spectrum upload");
    }
    g_kernels[key] = dev_ptr;
    *out = dev_ptr;
    return ok();
}

template <typename T>
cudaError_t dispatch(int n_b, const void* f, void* u, const void* kh, int64_t n, cudaStream_t st) {
    const auto* F = static_cast<const T*>(f);
    auto* U = static_cast<T*>(u);
    const auto* Kh = static_cast<const cx<T>*>(kh);
    switch (n_b) {
        case 4: return launch<T, 8, 4>(F, U, Kh, n, st);
        case 8: return launch<T, 16, 8>(F, U, Kh, n, st);
        case 16: return launch<T, 32, 16>(F, U, Kh, n, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace conv
}  // namespace lgf

using namespace lgf;

extern "C" lgf_status lgf_conv_blocks(const void* f_dev, void* u_dev, int64_t n_blocks, int32_t n_b,
                                      int32_t precision, void* stream) {
    if (!f_dev || !u_dev || n_blocks < 1 || n_blocks > (int64_t(1) << 31) - 1)
        return fail(LGF_ERR_INVALID_ARG, "lgf_conv_blocks: need f, u and 1 <= n_blocks < 2^31");
    if (n_b != 4 && n_b != 8 && n_b != 16) return fail(LGF_ERR_UNSUPPORTED, "lgf_conv_blocks: n_b must be 4, 8 or 16");
    if (precision != LGF_FP32 && precision != LGF_FP64)
        return fail(LGF_ERR_INVALID_ARG, "lgf_conv_blocks: precision must be LGF_FP32 or LGF_FP64");
    const size_t elem = precision == LGF_FP64 ? sizeof(double) : sizeof(float);
    const size_t bytes = size_t(n_blocks) * size_t(n_b) * n_b * n_b * elem;
    const auto* fb = static_cast<const unsigned char*>(f_dev);
    const auto* ub = static_cast<const unsigned char*>(u_dev);
    // a block is read whole before its output is written, by the same CTA:
    // f == u is allowed, any other overlap is not
    if (fb != ub && fb < ub + bytes && ub < fb + bytes)
        return fail(LGF_ERR_INVALID_ARG, "lgf_conv_blocks: f and u overlap (only f == u is allowed)");
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return conv::cuda_fail_conv(e, "cudaGetDevice");
    const void* kh = nullptr;
    lgf_status s = conv::kernel_for(device, n_b, precision, &kh);
    if (s != LGF_OK) return s;
    auto st = static_cast<cudaStream_t>(stream);
    e = precision == LGF_FP64 ? conv::dispatch<double>(n_b, f_dev, u_dev, kh, n_blocks, st)
                              : conv::dispatch<float>(n_b, f_dev, u_dev, kh, n_blocks, st);
    if (e != cudaSuccess) return conv::cuda_fail_conv(e, "launch");
    return ok();
}
