// In-register 1D DFTs for the padded block/interval FFTs (Sec. 2.2, the FFT
// and FFT^-1 steps of Eqs. alg_upfft and alg_dwfft).
//
// A line of length N lives in one thread's registers (cx<T> x[N]).  The
// transform is a compile-time mixed-radix decimation in time: N = R * M is R
// length-M transforms of the stride-R subsequences, then M radix-R butterflies
// with twiddles W_N^{r k1}.  Every index is a compile-time constant after
// unrolling, so twiddles are constant-bank operands and trivial twiddles
// (1, -1, +-i) cost nothing.  Zero padding is exploited explicitly: NZ is the
// number of leading inputs that may be non-zero, and subsequences that are all
// zero (or a single value) skip their arithmetic; floating-point rules forbid
// the compiler from dropping x*0 by itself.  Outputs a caller never reads are
// removed by dead-code elimination.
//
// W_TOP^j = exp(SIGN * 2 pi i j / TOP); SIGN = -1 forward, +1 inverse
// (unnormalised).  Twiddle tables hold cos/sin(2 pi j / S) for every supported
// top size S, filled from FP64 host values.
#pragma once

#include <cuda_runtime.h>

namespace lgf {
namespace dev {

template <typename T>
struct cx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> czero() {
    return {T(0), T(0)};
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) {
    return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) {
    return {a.x - b.x, a.y - b.y};
}
// acc + a*b (complex multiply-accumulate, four FMAs)
template <typename T>
__device__ __forceinline__ cx<T> cmac(cx<T> acc, cx<T> a, cx<T> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

// ---- twiddle tables ----
// every transform length S of the supported block sizes (level 0: 2 n_b;
// levels >= 1: the interval lengths)
constexpr int kTwSizes[] = {8, 10, 12, 16, 17, 18, 20, 24, 28, 32, 33, 34, 36, 40, 42};
constexpr int kTwCount = int(sizeof(kTwSizes) / sizeof(kTwSizes[0]));
// the i-th size of kTwSizes, usable in device code
__host__ __device__ constexpr int tw_size(int i) {
    constexpr int sizes[] = {8, 10, 12, 16, 17, 18, 20, 24, 28, 32, 33, 34, 36, 40, 42};
    return sizes[i];
}
// offset of size S in the tables: the sizes above, laid end to end (-1 if absent)
__host__ __device__ constexpr int tw_offset(int S) {
    int o = 0;
    for (int i = 0; i < kTwCount; ++i) {
        if (tw_size(i) == S) return o;
        o += tw_size(i);
    }
    return -1;
}
__host__ __device__ constexpr int tw_total() {
    int o = 0;
    for (int i = 0; i < kTwCount; ++i) o += tw_size(i);
    return o;
}
constexpr int kTwTotal = tw_total();

// One copy per translation unit (no relocatable device code); each TU fills
// its own copy through Launch<T>::init_twiddles.
static __constant__ double c_cos_d[kTwTotal];
static __constant__ double c_sin_d[kTwTotal];
static __constant__ float c_cos_f[kTwTotal];
static __constant__ float c_sin_f[kTwTotal];

template <typename T>
__device__ __forceinline__ T tw_cos(int i);
template <typename T>
__device__ __forceinline__ T tw_sin(int i);
template <>
__device__ __forceinline__ float tw_cos<float>(int i) { return c_cos_f[i]; }
template <>
__device__ __forceinline__ float tw_sin<float>(int i) { return c_sin_f[i]; }
template <>
__device__ __forceinline__ double tw_cos<double>(int i) { return c_cos_d[i]; }
template <>
__device__ __forceinline__ double tw_sin<double>(int i) { return c_sin_d[i]; }

// a * W_TOP^j
template <int TOP, int SIGN, typename T>
__device__ __forceinline__ cx<T> twmul(cx<T> a, int j) {
    j %= TOP;
    if (j < 0) j += TOP;
    if (j == 0) return a;
    if (2 * j == TOP) return {-a.x, -a.y};
    if (4 * j == TOP) return {T(-SIGN) * a.y, T(SIGN) * a.x};
    if (4 * j == 3 * TOP) return {T(SIGN) * a.y, T(-SIGN) * a.x};
    constexpr int kOff = tw_offset(TOP);
    static_assert(kOff >= 0, "transform length without a twiddle table");
    const T c = tw_cos<T>(kOff + j);
    const T s = T(SIGN) * tw_sin<T>(kOff + j);
    return {fma(a.x, c, -a.y * s), fma(a.x, s, a.y * c)};
}

__host__ __device__ constexpr int radix_of(int n) {
    if (n % 4 == 0 && n != 8) return 4;
    if (n % 2 == 0) return 2;
    for (int p = 3; p <= n; p += 2)
        if (n % p == 0) return p;
    return n;
}
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

// Radix-R DFT of z[0..R) in place, with z[r] = 0 for r >= RNZ (RNZ >= 1).
template <int TOP, int R, int SIGN, int RNZ, typename T>
__device__ __forceinline__ void butterfly(cx<T> (&z)[R]) {
    if constexpr (RNZ == 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) z[k] = z[0];
    } else if constexpr (R == 2) {
        const cx<T> a = z[0], b = z[1];
        z[0] = a + b;
        z[1] = a - b;
    } else if constexpr (R == 4) {
        const cx<T> a = z[0], b = z[1];
        const cx<T> t0 = RNZ > 2 ? a + z[2] : a;
        const cx<T> t1 = RNZ > 2 ? a - z[2] : a;
        const cx<T> t2 = RNZ > 3 ? b + z[3] : b;
        const cx<T> u = RNZ > 3 ? b - z[3] : b;
        const cx<T> t3 = {T(-SIGN) * u.y, T(SIGN) * u.x};   // (SIGN i) * u
        z[0] = t0 + t2;
        z[2] = t0 - t2;
        z[1] = t1 + t3;
        z[3] = t1 - t3;
    } else if constexpr (R == 3) {
        constexpr T h = T(0.86602540378443864676372317075293618);   // sqrt(3)/2
        const cx<T> a = z[0], b = z[1];
        const cx<T> c = RNZ > 2 ? z[2] : czero<T>();
        const cx<T> t1 = RNZ > 2 ? b + c : b;
        const cx<T> d = RNZ > 2 ? b - c : b;
        const cx<T> t2 = {fma(T(-0.5), t1.x, a.x), fma(T(-0.5), t1.y, a.y)};
        const cx<T> t3 = {T(-SIGN) * h * d.y, T(SIGN) * h * d.x};
        z[0] = a + t1;
        z[1] = t2 + t3;
        z[2] = t2 - t3;
    } else {
        // odd R >= 5: pair r with R-r so cos and sin factors are shared
        constexpr int H = (R - 1) / 2;
        cx<T> s[H + 1], d[H + 1];
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const bool a = r < RNZ, b = (R - r) < RNZ;
            s[r] = a ? (b ? z[r] + z[R - r] : z[r]) : (b ? z[R - r] : czero<T>());
            d[r] = a ? (b ? z[r] - z[R - r] : z[r]) : (b ? cx<T>{-z[R - r].x, -z[R - r].y} : czero<T>());
        }
        constexpr int kOff = tw_offset(TOP);
        static_assert(kOff >= 0, "transform length without a twiddle table");
        const cx<T> z0 = z[0];
        cx<T> out0 = z0;
#pragma unroll
        for (int r = 1; r <= H; ++r)
            if (r < RNZ || (R - r) < RNZ) out0 = out0 + s[r];
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            cx<T> P = z0, Q = czero<T>();
#pragma unroll
            for (int r = 1; r <= H; ++r) {
                if (!(r < RNZ || (R - r) < RNZ)) continue;
                const int m = (r * k) % R;
                const T c = tw_cos<T>(kOff + m * (TOP / R));
                const T sn = tw_sin<T>(kOff + m * (TOP / R));
                P.x = fma(s[r].x, c, P.x);
                P.y = fma(s[r].y, c, P.y);
                Q.x = fma(d[r].x, sn, Q.x);
                Q.y = fma(d[r].y, sn, Q.y);
            }
            // Z_k = P + SIGN i Q, Z_{R-k} = P - SIGN i Q
            z[k] = {P.x - T(SIGN) * Q.y, P.y + T(SIGN) * Q.x};
            z[R - k] = {P.x + T(SIGN) * Q.y, P.y - T(SIGN) * Q.x};
        }
        z[0] = out0;
    }
}

template <int TOP, int N, int SIGN, int NZ, typename T>
__device__ __forceinline__ void fft(cx<T> (&x)[N]);

template <int TOP, int M, int SIGN, int NZ, int R, int r, typename T>
__device__ __forceinline__ void sub_ffts(cx<T> (&y)[R][M]) {
    if constexpr (r < R) {
        constexpr int nzr = NZ > r ? (NZ - r + R - 1) / R : 0;
        fft<TOP, M, SIGN, cmin(nzr, M)>(y[r]);
        sub_ffts<TOP, M, SIGN, NZ, R, r + 1>(y);
    }
}

// x <- DFT_N(x) with twiddles of the top size TOP; inputs x[n >= NZ] are zero.
template <int TOP, int N, int SIGN, int NZ, typename T>
__device__ __forceinline__ void fft(cx<T> (&x)[N]) {
    if constexpr (N == 1) {
        if constexpr (NZ == 0) x[0] = czero<T>();
    } else if constexpr (NZ <= 1) {
#pragma unroll
        for (int k = 1; k < N; ++k) x[k] = NZ == 1 ? x[0] : czero<T>();
        if constexpr (NZ == 0) x[0] = czero<T>();
    } else {
        constexpr int R = radix_of(N);
        constexpr int M = N / R;
        cx<T> y[R][M];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int m = 0; m < M; ++m) y[r][m] = (r + R * m < NZ) ? x[r + R * m] : czero<T>();
        sub_ffts<TOP, M, SIGN, NZ, R, 0>(y);
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) {
            cx<T> z[R];
#pragma unroll
            for (int r = 0; r < R; ++r) z[r] = twmul<TOP, SIGN>(y[r][k1], r * k1 * (TOP / N));
            butterfly<TOP, R, SIGN, cmin(NZ, R)>(z);
#pragma unroll
            for (int k2 = 0; k2 < R; ++k2) x[k1 + M * k2] = z[k2];
        }
    }
}

}  // namespace dev
}  // namespace lgf
