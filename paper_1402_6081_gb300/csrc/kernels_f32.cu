// Instantiation of the solve kernels for T = float.
#include <cmath>

#include "kernels_impl.cuh"

namespace lgf {

template <>
cudaError_t Launch<float>::init_twiddles() {
    float c[dev::kTwTotal], s[dev::kTwTotal];
    for (int S : dev::kTwSizes) {
        const int o = dev::tw_offset(S);
        for (int j = 0; j < S; ++j) {
            const double a = 2.0 * M_PI * double(j) / double(S);
            c[o + j] = float(std::cos(a));
            s[o + j] = float(std::sin(a));
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(dev::c_cos_f, c, sizeof(c));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(dev::c_sin_f, s, sizeof(s));
    return e;
}

template struct Launch<float>;

// ---- persistent level-0 transforms (FP32) ----
bool cube_fft_supported(int S, int n) { return (S == 32 && n == 16) || (S == 16 && n == 8); }

template <int S, int N>
static cudaError_t cube_attrs(bool inverse, int n_sm, int* grid) {
    const size_t smem = inverse ? dev::c2r_cube_smem<S, N>() : dev::r2c_cube_smem<S, N>();
    const void* k = inverse ? reinterpret_cast<const void*>(dev::k_c2r_cube<S, N>)
                            : reinterpret_cast<const void*>(dev::k_r2c_cube<S, N>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, dev::cube_threads<S>(), smem);
    if (e != cudaSuccess) return e;
    *grid = n_sm * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

cudaError_t cube_fft_grid(int S, int n, bool inverse, int n_sm, int* grid) {
    if (S == 32 && n == 16) return cube_attrs<32, 16>(inverse, n_sm, grid);
    if (S == 16 && n == 8) return cube_attrs<16, 8>(inverse, n_sm, grid);
    return cudaErrorInvalidValue;
}

cudaError_t r2c_cube(int S, int n_in, const CUtensorMap& in_map, const R2CItem* items, int n, void* spec, int grid,
                     int* ctr, int* err, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const unsigned g = unsigned(grid < n ? grid : n);
    auto* out = static_cast<dev::cx<float>*>(spec);
#define LGF_R2C_CUBE(SS, NN)                                                                                    \
    if (S == SS && n_in == NN) {                                                                                 \
        dev::k_r2c_cube<SS, NN><<<g, dev::cube_threads<SS>(), dev::r2c_cube_smem<SS, NN>(), st>>>(in_map, items, \
                                                                                                 n, out, ctr,   \
                                                                                                 err);          \
        return cudaGetLastError();                                                                               \
    }
    LGF_R2C_CUBE(32, 16) LGF_R2C_CUBE(16, 8)
#undef LGF_R2C_CUBE
    return cudaErrorInvalidValue;
}

cudaError_t c2r_cube(int S, int n_out, const void* spec, const C2RItem* items, int n, float* dst, int64_t ds,
                     const float* add, int add_n, int64_t as, int grid, int* ctr, int* err, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const unsigned g = unsigned(grid < n ? grid : n);
    const auto* in = static_cast<const dev::cx<float>*>(spec);
#define LGF_C2R_CUBE(SS, NN)                                                                                       \
    if (S == SS && n_out == NN) {                                                                                   \
        dev::k_c2r_cube<SS, NN><<<g, dev::cube_threads<SS>(), dev::c2r_cube_smem<SS, NN>(), st>>>(                 \
            in, items, n, dst, ds, add, add_n, as, ctr, err);                                                      \
        return cudaGetLastError();                                                                                  \
    }
    LGF_C2R_CUBE(32, 16) LGF_C2R_CUBE(16, 8)
#undef LGF_C2R_CUBE
    return cudaErrorInvalidValue;
}

}  // namespace lgf
