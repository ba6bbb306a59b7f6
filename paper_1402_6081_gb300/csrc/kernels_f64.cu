// Instantiation of the solve kernels for T = double.
#include <cmath>

#include "kernels_impl.cuh"

namespace lgf {

template <>
cudaError_t Launch<double>::init_twiddles() {
    double c[dev::kTwTotal], s[dev::kTwTotal];
    for (int S : dev::kTwSizes) {
        const int o = dev::tw_offset(S);
        for (int j = 0; j < S; ++j) {
            const double a = 2.0 * M_PI * double(j) / double(S);
            c[o + j] = double(std::cos(a));
            s[o + j] = double(std::sin(a));
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(dev::c_cos_d, c, sizeof(c));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(dev::c_sin_d, s, sizeof(s));
    return e;
}

template struct Launch<double>;

}  // namespace lgf
