// Launchers of the block sizes n_b = 6, 10, 12, 14 (LaunchExt), templated on T;
// included by kernels_ext_f32.cu and kernels_ext_f64.cu.  Same kernels as the
// sizes 4, 8 and 16 (kernels_impl.cuh), other template arguments:
//   n_b   level-0 length S0 = 2 n_b   interval length S_I (>= 2 n_I - 1)   n_I
//    6          12                        16                                  7
//   10          20                        24                                 11
//   12          24                        28                                 13
//   14          28                        32                                 15
// Reg and Interp use the dense 1D products (every stencil order).
#pragma once

#include <cmath>

#include "kernels_impl.cuh"

namespace lgf {

template <typename T>
cudaError_t LaunchExt<T>::init_twiddles() {
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

template <typename T>
cudaError_t LaunchExt<T>::r2c(int S, int n_in, const T* src, int64_t stride, const R2CItem* items, int n,
                              void* spec, cudaStream_t st) {
#define LGF_R2C(SS, NN) \
    if (S == SS && n_in == NN) return launch_r2c<T, SS, NN>(src, stride, items, n, spec, st);
    LGF_R2C(12, 6) LGF_R2C(20, 10) LGF_R2C(24, 12) LGF_R2C(28, 14)     // level 0
    LGF_R2C(16, 7) LGF_R2C(24, 11) LGF_R2C(28, 13) LGF_R2C(32, 15)     // intervals
    LGF_R2C(16, 6) LGF_R2C(24, 10) LGF_R2C(28, 12) LGF_R2C(32, 14)     // level 1 from the blocks
#undef LGF_R2C
    if constexpr (sizeof(T) == 4) return r2c_large(S, n_in, src, stride, items, n, spec, st);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t LaunchExt<T>::c2r(int S, int n_out, const void* spec, const C2RItem* items, int n, T* dst, int64_t ds,
                              const T* add, int add_n, int64_t as, cudaStream_t st) {
#define LGF_C2R(SS, NN) \
    if (S == SS && n_out == NN) return launch_c2r<T, SS, NN>(spec, items, n, dst, ds, add, add_n, as, st);
    LGF_C2R(12, 6) LGF_C2R(20, 10) LGF_C2R(24, 12) LGF_C2R(28, 14)
    LGF_C2R(16, 7) LGF_C2R(24, 11) LGF_C2R(28, 13) LGF_C2R(32, 15)
#undef LGF_C2R
    if constexpr (sizeof(T) == 4) return c2r_large(S, n_out, spec, items, n, dst, ds, add, add_n, as, st);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t LaunchExt<T>::mac_interval(const void* fh, const void* kh, void* uh, const int* gnbr, const int* order,
                                       int n_groups, int S, int variant, int include_self, const CUtensorMap* tmap,
                                       int* err, cudaStream_t st, int oct, int gpc) {
    // the two-frequency and paired variants stay with the sizes 4, 8, 16
    const int v = variant == 2 || variant == 3 ? 1 : variant;
    switch (S) {
        case 12: return launch_mac_interval<T, 12>(fh, kh, uh, gnbr, order, n_groups, v, include_self, tmap, err, st, oct, gpc);
        case 20: return launch_mac_interval<T, 20>(fh, kh, uh, gnbr, order, n_groups, v, include_self, tmap, err, st, oct, gpc);
        case 24: return launch_mac_interval<T, 24>(fh, kh, uh, gnbr, order, n_groups, v, include_self, tmap, err, st, oct, gpc);
        case 28: return launch_mac_interval<T, 28>(fh, kh, uh, gnbr, order, n_groups, v, include_self, tmap, err, st, oct, gpc);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t LaunchExt<T>::mac_persist(const void* fh, const void* kh, void* uh, const PersistPlan& pp, int S,
                                      int early, cudaStream_t st) {
    if constexpr (sizeof(T) != 4) {
        return cudaErrorInvalidValue;
    } else {
        switch (S) {
            case 12: return launch_mac_persist_form<12>(fh, kh, uh, pp, early, st);
            case 20: return launch_mac_persist_form<20>(fh, kh, uh, pp, early, st);
            case 24: return launch_mac_persist_form<24>(fh, kh, uh, pp, early, st);
            case 28: return launch_mac_persist_form<28>(fh, kh, uh, pp, early, st);
            default: return mac_persist_large(fh, kh, uh, pp, S, early, st);
        }
    }
}

template <typename T>
cudaError_t LaunchExt<T>::reg(int n_b, int n_max, const T* child_src, int child_is_block, const int* child_index,
                              const int* parent_slot, int n_parents, T* dst, const T* W, int comp, cudaStream_t st) {
    (void)n_max;
    if (n_parents == 0) return cudaSuccess;
#define LGF_REG(NI) \
    if (n_b + 1 == NI) return launch_reg<T, NI, 0>(child_src, child_is_block, child_index, parent_slot, n_parents, dst, W, comp, st);
    LGF_REG(7) LGF_REG(11) LGF_REG(13) LGF_REG(15)
#undef LGF_REG
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t LaunchExt<T>::interp(int n_b, int n_max, const int* slot, const int* parent, int n_items, T* u,
                                 const T* up, const T* W, int accumulate, const int* block, int comp,
                                 cudaStream_t st) {
    (void)n_max;
    if (n_items == 0) return cudaSuccess;
#define LGF_INTERP(NI)                                                                                        \
    if (n_b + 1 == NI) {                                                                                      \
        auto kern = comp ? dev::k_interp<T, NI, sizeof(T) == 4, 0> : dev::k_interp<T, NI, false, 0>;            \
        kern<<<n_items, dev::kLineThreads, 0, st>>>(slot, parent, u, up, pack_w<T, NI>(W), accumulate, block); \
        return cudaGetLastError();                                                                            \
    }
    LGF_INTERP(7) LGF_INTERP(11) LGF_INTERP(13) LGF_INTERP(15)
#undef LGF_INTERP
    return cudaErrorInvalidValue;
}

}  // namespace lgf
