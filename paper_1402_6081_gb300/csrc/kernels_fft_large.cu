// Per-block transforms (the in-shared-memory kernels of kernels_impl.cuh) for
// the FP32 block sizes 18 and 20, whose cubes still fit a CTA's shared memory:
//   n_b   level 0 (S0, n)   intervals (S_I, n_I)   level 1 from the blocks
//   18      36, 18            40, 19                 40, 18
//   20      40, 20            42, 21                 42, 20
// (largest: the 42-point interval cube, 155 KB plus the 37 KB staged input).
// The other steps of these sizes, and every FP64 step, run the run-time-size
// kernels of generic.cu.  This unit has its own copy of the twiddle tables.
#include <cmath>

#include "kernels_impl.cuh"

namespace lgf {

bool fft_large_supported(int S, int n) {
    return (S == 36 && n == 18) || (S == 40 && (n == 18 || n == 19 || n == 20)) || (S == 42 && (n == 20 || n == 21));
}

cudaError_t fft_large_init_twiddles() {
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
    return e == cudaSuccess ? cudaMemcpyToSymbol(dev::c_sin_f, s, sizeof(s)) : e;
}

cudaError_t r2c_large(int S, int n_in, const float* src, int64_t stride, const R2CItem* items, int n, void* spec,
                      cudaStream_t st) {
#define LGF_R2C(SS, NN) \
    if (S == SS && n_in == NN) return launch_r2c<float, SS, NN>(src, stride, items, n, spec, st);
    LGF_R2C(36, 18) LGF_R2C(40, 19) LGF_R2C(40, 18) LGF_R2C(40, 20) LGF_R2C(42, 21) LGF_R2C(42, 20)
#undef LGF_R2C
    return cudaErrorInvalidValue;
}

cudaError_t c2r_large(int S, int n_out, const void* spec, const C2RItem* items, int n, float* dst, int64_t ds,
                      const float* add, int add_n, int64_t as, cudaStream_t st) {
#define LGF_C2R(SS, NN) \
    if (S == SS && n_out == NN) return launch_c2r<float, SS, NN>(spec, items, n, dst, ds, add, add_n, as, st);
    LGF_C2R(36, 18) LGF_C2R(40, 19) LGF_C2R(40, 20) LGF_C2R(42, 21)
#undef LGF_C2R
    return cudaErrorInvalidValue;
}

}  // namespace lgf
