// Isolated-block solves that allocate no device memory (lgf_solve_blocks_noalloc).
//
// Some callers cannot allocate device memory while they run: code inside a
// host-side allocator hook, a real-time loop whose memory was fixed up front,
// or a framework that owns the whole device heap and forbids cudaMalloc.  This
// entry point gives them the single-block FFT convolution of the solver with
// all of its working memory in one file-scope device array: the forward
// spectra of the blocks (overwritten in place by the products), the kernel
// spectrum of each supported (n_b, precision), and the launch item tables.
//
// The array is kNoAllocScratchBytes (32 MiB) on every GPU that loads this
// library and stays until the process exits.  In host code its name is only a
// host-side stand-in, so the device address is fetched once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device; that first call also uploads the item tables, the FFT twiddles
// of this translation unit and the kernel spectra of all six (n_b, precision)
// pairs (under 0.5 MiB together), with synchronous copies.  Make the first
// call on each device before any stream capture.  Later calls, whatever their
// n_b and precision, only launch three kernels on the given stream.
//
// All calls share the array and it keeps the last call's contents; every
// value a call reads is written earlier in the same call, so nothing needs
// clearing.  Two calls whose kernels overlap on the GPU (different streams,
// or different host threads) overwrite each other's spectra: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <vector>

#include "kernels_impl.cuh"

namespace lgf {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr size_t kKernelRegion = size_t(1) << 20;      // kernel spectra, fixed offsets
constexpr int kMaxItems = 4096;
constexpr size_t kItemRegion = size_t(128) << 10;      // identity R2C / C2R items
constexpr size_t kSpecOffset = kKernelRegion + kItemRegion;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

int nb_index(int n_b) { return n_b == 4 ? 0 : n_b == 8 ? 1 : n_b == 16 ? 2 : -1; }

// byte offset of the kernel spectrum of (n_b, precision) inside the kernel region
size_t kernel_offset(int n_b, int prec) {
    size_t off = 0;
    for (int nb : {4, 8, 16})
        for (int pr : {LGF_FP32, LGF_FP64}) {
            if (nb == n_b && pr == prec) return off;
            const size_t bytes = size_t(nw_of(2 * nb)) * 2 * (pr == LGF_FP64 ? 8 : 4);
            off += (bytes + 255) / 256 * 256;
        }
    return off;
}

struct DeviceState {
    unsigned char* base = nullptr;
};
std::mutex g_mu;
std::map<int, DeviceState> g_state;

lgf_status cuda_err(cudaError_t e, const char* what) {
    return fail(LGF_ERR_CUDA, std::string("lgf_solve_blocks_noalloc: ") + what + ": " + cudaGetErrorString(e));
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

// Kernel spectrum of the block with itself (offset d = 0, level 0), FP64 on the
// host, rounded to the precision, copied into the kernel region.
lgf_status load_kernel(unsigned char* base, int n_b, int prec) {
    const int S = 2 * n_b;
    const int64_t NW = nw_of(S);
    auto tab = green_abs_table(1, n_b - 1);
    std::vector<std::complex<double>> kh(static_cast<size_t>(NW));
    const int d[3] = {0, 0, 0};
    kernel_spectrum(n_b, n_b, 1, S, d, tab->data(), n_b - 1, kh.data());
    cudaError_t e;
    unsigned char* dst = base + kernel_offset(n_b, prec);
    if (prec == LGF_FP64) {
        e = cudaMemcpy(dst, kh.data(), sizeof(double) * 2 * size_t(NW), cudaMemcpyHostToDevice);
    } else {
        std::vector<float> f(2 * size_t(NW));
        for (size_t i = 0; i < size_t(NW); ++i) {
            f[2 * i] = float(kh[i].real());
            f[2 * i + 1] = float(kh[i].imag());
        }
        e = cudaMemcpy(dst, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return cuda_err(e, "kernel spectrum upload");
    return ok();
}

// First call on a device: the array's device address, item tables, twiddles
// and every kernel spectrum.
lgf_status setup_device(int device, DeviceState& st) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress");
    std::vector<R2CItem> r(kMaxItems);
    std::vector<C2RItem> c(kMaxItems);
    for (int i = 0; i < kMaxItems; ++i) {
        r[size_t(i)] = {i, i};
        c[size_t(i)] = {i, i, -1};
    }
    unsigned char* base = static_cast<unsigned char*>(ptr);
    if ((e = cudaMemcpy(base + kKernelRegion, r.data(), sizeof(R2CItem) * r.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_err(e, "item upload");
    if ((e = cudaMemcpy(base + kKernelRegion + sizeof(R2CItem) * kMaxItems, c.data(),
                        sizeof(C2RItem) * c.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_err(e, "item upload");
    if ((e = upload_twiddles<float>()) != cudaSuccess) return cuda_err(e, "twiddle upload");
    if ((e = upload_twiddles<double>()) != cudaSuccess) return cuda_err(e, "twiddle upload");
    for (int nb : {4, 8, 16})
        for (int pr : {LGF_FP32, LGF_FP64}) {
            lgf_status r = load_kernel(base, nb, pr);
            if (r != LGF_OK) return r;
        }
    st.base = base;
    (void)device;
    return ok();
}

// spec[b][w] <- spec[b][w] * kh[w] (the single product of Eq. alg_mult for a
// block whose only near neighbour is itself)
// (block spectra are NWS apart; entries past NW are padding and stay as they are)
template <typename T>
__global__ void k_mul_spectrum(dev::cx<T>* __restrict__ spec, const dev::cx<T>* __restrict__ kh, int64_t NW,
                               int64_t NWS, int64_t total) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t w = i % NWS;
        if (w >= NW) continue;
        const dev::cx<T> f = spec[i];
        spec[i] = dev::cmac(dev::czero<T>(), f, dev::ldg_cx(kh + w));
    }
}

template <typename T, int S, int NB>
lgf_status run(DeviceState& st, const T* f, T* u, int64_t n, int prec, cudaStream_t stream) {
    const int64_t NW = nw_of(S), NWS = nws_of(S);
    auto* spec = reinterpret_cast<dev::cx<T>*>(st.base + kSpecOffset);
    const auto* kh = reinterpret_cast<const dev::cx<T>*>(st.base + kernel_offset(NB, prec));
    const auto* r2c = reinterpret_cast<const R2CItem*>(st.base + kKernelRegion);
    const auto* c2r = reinterpret_cast<const C2RItem*>(st.base + kKernelRegion + sizeof(R2CItem) * kMaxItems);
    const int64_t b3 = int64_t(NB) * NB * NB;
    cudaError_t e = launch_r2c<T, S, NB>(f, b3, r2c, int(n), spec, stream);
    if (e != cudaSuccess) return cuda_err(e, "forward FFT");
    const int64_t total = n * NWS;
    const int grid = int(std::min<int64_t>((total + 255) / 256, 152 * 16));
    k_mul_spectrum<T><<<grid, 256, 0, stream>>>(spec, kh, NW, NWS, total);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "spectral product");
    e = launch_c2r<T, S, NB>(spec, c2r, int(n), u, b3, nullptr, 0, 0, stream);
    if (e != cudaSuccess) return cuda_err(e, "inverse FFT");
    return ok();
}

}  // namespace
}  // namespace lgf

using namespace lgf;

extern "C" lgf_status lgf_noalloc_max_blocks(int32_t n_b, int32_t precision, int64_t* max_blocks) {
    if (!max_blocks || nb_index(n_b) < 0 || (precision != LGF_FP32 && precision != LGF_FP64))
        return fail(LGF_ERR_INVALID_ARG, "lgf_noalloc_max_blocks: need n_b in {4, 8, 16}, a precision and an output");
    const size_t per = size_t(nws_of(2 * n_b)) * 2 * (precision == LGF_FP64 ? 8 : 4);
    *max_blocks = std::min<int64_t>(kMaxItems, int64_t((kNoAllocScratchBytes - kSpecOffset) / per));
    return ok();
}

extern "C" lgf_status lgf_solve_blocks_noalloc(const void* f_dev, void* u_dev, int64_t n_blocks, int32_t n_b,
                                               int32_t precision, void* stream) {
    if (!f_dev || !u_dev || n_blocks < 1)
        return fail(LGF_ERR_INVALID_ARG, "lgf_solve_blocks_noalloc: need f, u and n_blocks >= 1");
    if (nb_index(n_b) < 0) return fail(LGF_ERR_UNSUPPORTED, "lgf_solve_blocks_noalloc: n_b must be 4, 8 or 16");
    if (precision != LGF_FP32 && precision != LGF_FP64)
        return fail(LGF_ERR_INVALID_ARG, "lgf_solve_blocks_noalloc: precision must be LGF_FP32 or LGF_FP64");
    int64_t mx = 0;
    lgf_noalloc_max_blocks(n_b, precision, &mx);
    if (n_blocks > mx)
        return fail(LGF_ERR_INVALID_ARG, "lgf_solve_blocks_noalloc: " + std::to_string(n_blocks) +
                                             " blocks exceed the limit of " + std::to_string(mx) +
                                             " for n_b = " + std::to_string(n_b) + " in this precision (" +
                                             std::to_string(kNoAllocScratchBytes >> 20) + " MiB scratch)");
    {
        // the inverse transforms write u while later blocks' sources are
        // still to be read: the byte ranges of f and u must be disjoint
        const uintptr_t bytes = uintptr_t(n_blocks) * uintptr_t(n_b) * n_b * n_b * (precision == LGF_FP64 ? 8 : 4);
        const uintptr_t f0 = reinterpret_cast<uintptr_t>(f_dev), u0 = reinterpret_cast<uintptr_t>(u_dev);
        if (f0 < u0 + bytes && u0 < f0 + bytes)
            return fail(LGF_ERR_INVALID_ARG, "lgf_solve_blocks_noalloc: f and u must not overlap");
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
    DeviceState* st = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        DeviceState& s = g_state[device];
        if (!s.base) {
            lgf_status r = setup_device(device, s);
            if (r != LGF_OK) return r;
        }
        st = &s;
    }
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    if (precision == LGF_FP64) {
        const auto* f = static_cast<const double*>(f_dev);
        auto* u = static_cast<double*>(u_dev);
        if (n_b == 4) return run<double, 8, 4>(*st, f, u, n_blocks, precision, strm);
        if (n_b == 8) return run<double, 16, 8>(*st, f, u, n_blocks, precision, strm);
        return run<double, 32, 16>(*st, f, u, n_blocks, precision, strm);
    }
    const auto* f = static_cast<const float*>(f_dev);
    auto* u = static_cast<float*>(u_dev);
    if (n_b == 4) return run<float, 8, 4>(*st, f, u, n_blocks, precision, strm);
    if (n_b == 8) return run<float, 16, 8>(*st, f, u, n_blocks, precision, strm);
    return run<float, 32, 16>(*st, f, u, n_blocks, precision, strm);
}
