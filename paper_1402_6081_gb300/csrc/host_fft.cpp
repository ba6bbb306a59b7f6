// Host FP64 complex FFT for the plan-time kernel spectra (Eq. precomp).
// Recursive mixed-radix decimation in time: a length n = r * m transform is r
// transforms of length m on the stride-r subsequences, combined with twiddles
// W_n^{j k1} and a radix-r DFT; r is the smallest prime factor of n.  Roots of
// unity come from one table per call (lengths up to 96).
#include <cmath>
#include <complex>
#include <vector>

#include "lgf_internal.h"

namespace lgf {
namespace {

using cd = std::complex<double>;
constexpr int kMaxN = 96;

int smallest_factor(int n) {
    if (n % 2 == 0) return 2;
    for (int p = 3; p * p <= n; p += 2)
        if (n % p == 0) return p;
    return n;
}

// W[j] = exp(sign 2 pi i j / ntop); W_n^k = W[k * (ntop / n) mod ntop]
void rec(const cd* in, int is, cd* out, int n, const cd* W, int ntop) {
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    const int r = smallest_factor(n);
    const int m = n / r;
    cd y[kMaxN];
    for (int j = 0; j < r; ++j) rec(in + size_t(j) * is, is * r, y + j * m, m, W, ntop);
    const int step = ntop / n, rstep = ntop / r;
    cd t[kMaxN];
    for (int k1 = 0; k1 < m; ++k1) {
        for (int j = 0; j < r; ++j) t[j] = y[j * m + k1] * W[(j * k1 * step) % ntop];
        for (int k2 = 0; k2 < r; ++k2) {
            cd s = 0.0;
            for (int j = 0; j < r; ++j) s += t[j] * W[((j * k2) % r) * rstep];
            out[k1 + m * k2] = s;
        }
    }
}

}  // namespace

void fft_lines(std::complex<double>* base, int n, int stride, int count, int64_t line_stride,
               int sign) {
    cd W[kMaxN];
    for (int j = 0; j < n; ++j) {
        const double a = 2.0 * M_PI * double(j) / double(n);
        W[j] = cd(std::cos(a), sign * std::sin(a));
    }
    cd in[kMaxN], out[kMaxN];
    for (int c = 0; c < count; ++c) {
        cd* x = base + c * line_stride;
        for (int i = 0; i < n; ++i) in[i] = x[size_t(i) * stride];
        rec(in, 1, out, n, W, n);
        for (int i = 0; i < n; ++i) x[size_t(i) * stride] = out[i];
    }
}

void fft_inplace(std::complex<double>* x, int n, int stride, int sign) {
    fft_lines(x, n, stride, 1, 0, sign);
}

}  // namespace lgf
