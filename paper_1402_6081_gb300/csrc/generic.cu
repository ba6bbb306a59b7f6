// Solve kernels for the block sizes that the per-block, in-shared-memory
// kernels cannot hold (even n_b of [18, 32]): the same steps of Sec. 3.1 with
// every size a run-time argument.
//
//  * Transforms (Eqs. alg_upfft, alg_dwfft): one axis per launch, between the
//    level's spectrum buffer and a scratch indexed by item that holds only
//    the planes a zero-padded line can reach, each output value of a line the
//    plain DFT sum over its non-zero inputs (at most n of the S samples are
//    non-zero along an axis: zero padding), with the twiddles of a table
//    filled from FP64 host values.  Consecutive threads take consecutive kx,
//    so every pass reads and writes whole 32-value runs.
//  * Products (Eq. alg_mult): a CTA per chunk of 32 frequencies and range of
//    target sibling groups, the chunk's 343 coefficient rows staged once in
//    shared memory from the half table, a warp per group at a time with the
//    8 x 8 sibling products of each neighbour group in registers (mac_block).
//  * Reg and Interp (Eqs. alg_reg, alg_interp): the three axis passes of an
//    item in shared memory (a per-CTA scratch in global memory when the cubes
//    do not fit), each sum over its row's band of the stencil matrix;
//    compensated FP32 sums where asked.  Reg runs a CTA per (parent, child)
//    for the x and y passes and sums the children in its z pass.
#include <algorithm>

#include "kernels_impl.cuh"

namespace lgf {
namespace gen {

using dev::cx;
using dev::czero;
using dev::ldg_cx;

constexpr int kThreads = 256;
constexpr int kLineThreads = 128;   // lines per CTA of the y / z passes
constexpr int kRiThreads = 512;     // threads per Reg / Interp CTA

// (cos, sign sin)(2 pi m / S), m < S, into shared memory
template <typename T>
__device__ __forceinline__ void load_twiddles(cx<T>* tw_s, const cx<T>* __restrict__ twt, int S, int sign) {
    for (int m = threadIdx.x; m < S; m += blockDim.x) {
        const cx<T> w = ldg_cx(twt + m);
        tw_s[m] = {w.x, T(sign) * w.y};
    }
}
__device__ __forceinline__ int wrap(int i, int S) { return i >= S ? i - S : i; }

// ---- forward transform, x: real rows of the input to the first NX values.
// The N^2 NX outputs (row, k) of an item, k fastest, are cut into `tiles`
// tiles of tile_len; a CTA stages its tile's rows in shared memory and then
// computes kXTile / kThreads outputs per thread, the twiddle index (x k mod S)
// advanced by k per term.
constexpr int kXTile = 4 * kThreads;

template <typename T>
__global__ void __launch_bounds__(kThreads) g_r2c_x(const T* __restrict__ src, int64_t stride,
                                                    const R2CItem* __restrict__ items, int tiles, int tile_len,
                                                    cx<T>* __restrict__ A, int64_t nws, int S, int N,
                                                    const cx<T>* __restrict__ twt) {
    extern __shared__ __align__(16) unsigned char g_smem[];
    cx<T>* tw_s = reinterpret_cast<cx<T>*>(g_smem);
    T* rows = reinterpret_cast<T*>(tw_s + S);   // [rows of this tile][N]
    const int NX = S / 2 + 1, per_item = N * N * NX;
    const int it = blockIdx.x / tiles, j0 = (blockIdx.x % tiles) * tile_len;
    const int j1 = min(j0 + tile_len, per_item);
    const int row0 = j0 / NX, row1 = (j1 - 1) / NX + 1;
    const R2CItem item = items[it];
    const T* in = src + int64_t(item.src) * stride + int64_t(row0) * N;
    load_twiddles(tw_s, twt, S, -1);
    for (int q = threadIdx.x; q < (row1 - row0) * N; q += blockDim.x) rows[q] = __ldg(in + q);
    __syncthreads();
    cx<T>* out = A + int64_t(item.dst) * nws;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const int k = j % NX, row = j / NX;
        const T* v = rows + (row - row0) * N;
        cx<T> acc = czero<T>();
        int idx = 0;
        for (int x = 0; x < N; ++x) {
            const cx<T> w = tw_s[idx];
            acc.x = fma(v[x], w.x, acc.x);
            acc.y = fma(v[x], w.y, acc.y);
            idx = wrap(idx + k, S);
        }
        const int y = row % N, z = row / N;
        out[(z * S + y) * NX + k] = acc;
    }
}

// ---- one complex axis (y: stride NX, planes z < N; z: stride S NX, all y)
// out[j] = sum_{m < nin} in[m] exp(sign i 2 pi j m / S), j < nout.  A side
// with slots addresses item it at slots[it * slot_stride] * its stride (the
// level's spectrum buffer), one without at it * its stride (the transform
// scratch, whose items hold only the planes the other passes use).  Thread
// per line (item, other, kx), kx fastest so the loads and stores of a warp are
// contiguous; the line's inputs are staged in shared memory (column per
// thread) and every output sums them against warp-uniform twiddles, two
// outputs per trip.
template <typename T>
__global__ void __launch_bounds__(kLineThreads) g_axis(const cx<T>* __restrict__ in,
                                                       const int* __restrict__ in_slots, int64_t in_ws,
                                                       cx<T>* __restrict__ out, const int* __restrict__ out_slots,
                                                       int64_t out_ws, int slot_stride, int n_items, int S, int nin,
                                                       int nout, int n_other, int64_t axis_stride,
                                                       int64_t other_stride, int sign,
                                                       const cx<T>* __restrict__ twt) {
    extern __shared__ __align__(16) unsigned char g_smem[];
    cx<T>* tw_s = reinterpret_cast<cx<T>*>(g_smem);
    cx<T>* col = tw_s + S + threadIdx.x;        // [nin][blockDim.x], this thread's column
    load_twiddles(tw_s, twt, S, sign);
    __syncthreads();
    const int NX = S / 2 + 1;
    const int64_t lines = int64_t(n_items) * n_other * NX;
    const int64_t L = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (L >= lines) return;
    const int kx = int(L % NX);
    const int64_t t = L / NX;
    const int o = int(t % n_other), it = int(t / n_other);
    const int64_t line = int64_t(o) * other_stride + kx;
    const int64_t ib = (in_slots ? int64_t(in_slots[int64_t(it) * slot_stride]) : int64_t(it)) * in_ws + line;
    const int64_t ob = (out_slots ? int64_t(out_slots[int64_t(it) * slot_stride]) : int64_t(it)) * out_ws + line;
    for (int m = 0; m < nin; ++m) col[m * blockDim.x] = ldg_cx(in + ib + int64_t(m) * axis_stride);
    for (int j = 0; j < nout; j += 2) {
        const int j1 = j + 1 < S ? j + 1 : 0;
        cx<T> a0 = czero<T>(), a1 = czero<T>();
        int i0 = 0, i1 = 0;
        for (int m = 0; m < nin; ++m) {
            const cx<T> v = col[m * blockDim.x];
            const cx<T> w0 = tw_s[i0], w1 = tw_s[i1];
            a0.x = fma(v.x, w0.x, fma(-v.y, w0.y, a0.x));
            a0.y = fma(v.x, w0.y, fma(v.y, w0.x, a0.y));
            a1.x = fma(v.x, w1.x, fma(-v.y, w1.y, a1.x));
            a1.y = fma(v.x, w1.y, fma(v.y, w1.x, a1.y));
            i0 = wrap(i0 + j, S);
            i1 = wrap(i1 + j1, S);
        }
        out[ob + int64_t(j) * axis_stride] = a0;
        if (j + 1 < nout) out[ob + int64_t(j + 1) * axis_stride] = a1;
    }
}

// ---- inverse transform, x: Hermitian rows to the first N real samples (+ add).
// The N^3 outputs (row, x) of an item, x fastest, cut into tiles as above; a
// CTA stages its tile's rows of NX values in shared memory.
template <typename T>
__global__ void __launch_bounds__(kThreads) g_c2r_x(const cx<T>* __restrict__ U, const C2RItem* __restrict__ items,
                                                    int tiles, int tile_len, T* __restrict__ dst, int64_t dst_stride,
                                                    const T* __restrict__ add, int add_n, int64_t add_stride,
                                                    int64_t nws, int S, int N, const cx<T>* __restrict__ twt) {
    extern __shared__ __align__(16) unsigned char g_smem[];
    cx<T>* tw_s = reinterpret_cast<cx<T>*>(g_smem);
    const int NX = S / 2 + 1, per_item = N * N * N;
    cx<T>* rows = tw_s + S;                     // [rows of this tile][NX]
    const int it = blockIdx.x / tiles, j0 = (blockIdx.x % tiles) * tile_len;
    const int j1 = min(j0 + tile_len, per_item);
    const int row0 = j0 / N, row1 = (j1 - 1) / N + 1;
    const C2RItem item = items[it];
    const cx<T>* in = U + int64_t(item.src) * nws;
    load_twiddles(tw_s, twt, S, +1);
    for (int q = threadIdx.x; q < (row1 - row0) * NX; q += blockDim.x) {
        const int row = row0 + q / NX, k = q % NX;
        rows[q] = ldg_cx(in + ((row / N) * S + row % N) * NX + k);
    }
    __syncthreads();
    T* out = dst + int64_t(item.dst) * dst_stride;
    const T* ad = (add != nullptr && item.aux >= 0) ? add + int64_t(item.aux) * add_stride : nullptr;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const int x = j % N, row = j / N;
        const cx<T>* X = rows + (row - row0) * NX;
        // x[n] = X[0] + 2 sum_{0 < k < S/2} Re(X[k] e^{+i 2 pi n k / S}) + X[S/2] (-1)^n (S even)
        T acc = X[0].x;
        const int kmax = (S % 2 == 0) ? S / 2 : NX;
        int idx = wrap(x, S);
        for (int k = 1; k < kmax; ++k) {
            const cx<T> w = tw_s[idx];
            acc += T(2) * (X[k].x * w.x - X[k].y * w.y);
            idx = wrap(idx + x, S);
        }
        if (S % 2 == 0) acc += ((x & 1) ? T(-1) : T(1)) * X[S / 2].x;
        const int y = row % N, z = row / N;
        if (ad) acc += __ldg(ad + (z * add_n + y) * add_n + x);
        out[row * N + x] = acc;
    }
}

// ---- products: a CTA per (group range, chunk of 32 frequencies); the
// chunk's 343 coefficient rows are staged once, then its 8 warps take the
// range's groups in turn (warp w: groups g0 + w, g0 + w + 8, ...).
template <typename T>
__global__ void __launch_bounds__(256) g_mac(const cx<T>* __restrict__ fh, const cx<T>* __restrict__ kh,
                                             cx<T>* __restrict__ uh, const int* __restrict__ gnbr, int n_groups,
                                             int groups_per_cta, int include_self, int64_t nw, int64_t nws) {
    extern __shared__ __align__(16) unsigned char g_smem[];
    cx<T>* sk = reinterpret_cast<cx<T>*>(g_smem);   // [343][32]
    const int64_t w0 = int64_t(blockIdx.y) * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    // rows 171..342 stored; row d < 171 is the conjugate of row 342 - d
    for (int i = tid; i < 343 * 32; i += 256) {
        const int d = i >> 5;
        const int64_t w = w0 + (i & 31);
        cx<T> v = czero<T>();
        if (w < nw) v = d >= 171 ? ldg_cx(kh + int64_t(d - 171) * nws + w) : dev::conjx(ldg_cx(kh + int64_t(171 - d) * nws + w));
        sk[i] = v;
    }
    __syncthreads();
    const int64_t w = w0 + threadIdx.x;
    const int64_t wc = w < nw ? w : nw - 1;
    const int g0 = blockIdx.x * groups_per_cta, g1 = min(g0 + groups_per_cta, n_groups);
    for (int g = g0 + int(threadIdx.y); g < g1; g += 8) {
        cx<T> acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = czero<T>();
        for (int e = 0; e < 27; ++e) {
            if (e == 13 && !include_self) continue;
            const int q = __ldg(gnbr + int64_t(g) * 27 + e);
            if (q < 0) continue;
            cx<T> F[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) F[c] = ldg_cx(fh + (int64_t(q) * 8 + c) * nws + wc);
            dev::mac_block(acc, F, sk, e);
        }
        if (w < nw) {
#pragma unroll
            for (int c = 0; c < 8; ++c) uh[(int64_t(g) * 8 + c) * nws + w] = acc[c];
        }
    }
}

// ---- Reg and Interp: one 1D pass over a cube, value (i along the axis) =
// sum_k M(i, k) in[k along the axis], M(i, k) = W[c][i][k] (interpolation) or
// W[c][k][i] (its adjoint).  Every row of M is non-zero on one contiguous band
// of k (the n_max nearest nodes of a point, or for the adjoint the points
// whose stencils hold a node), found once per CTA (band[c][i] = lo | hi << 16).
template <typename T>
struct Sum {
    T s = T(0), e = T(0);
    __device__ __forceinline__ void add(T w, T x, bool comp) {
        if constexpr (sizeof(T) == 4) {
            if (comp) {
                dev::acc_comp(s, e, w, x);
                return;
            }
        }
        s = fma(w, x, s);
    }
    __device__ __forceinline__ T get() const { return s + e; }
};

// W (2 x n x n) and the bands of M for both children into shared memory
template <typename T>
__device__ void load_stencil(T* W_s, int* band, const T* __restrict__ W, int n, bool adjoint) {
    for (int i = threadIdx.x; i < 2 * n * n; i += blockDim.x) W_s[i] = __ldg(W + i);
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * n; q += blockDim.x) {
        const int c = q / n, i = q % n;
        const T* Wc = W_s + c * n * n;
        int lo = n, hi = 0;
        for (int k = 0; k < n; ++k)
            if ((adjoint ? Wc[k * n + i] : Wc[i * n + k]) != T(0)) {
                lo = min(lo, k);
                hi = k + 1;
            }
        band[q] = lo < hi ? (lo | (hi << 16)) : 0;
    }
    __syncthreads();
}

// axis a of a cube of edge n (in: edge in_n <= n, zero beyond); emit(i, value).
// Plain sums alternate two partial sums (two chains in flight).
template <typename T, typename Emit>
__device__ __forceinline__ void pass(const T* in, int in_n, int n, int axis, const T* Wc, const int* band,
                                     bool adjoint, bool comp, Emit emit) {
    const int n3 = n * n * n;
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int x = i % n, y = (i / n) % n, z = i / (n * n);
        const int o = axis == 0 ? x : axis == 1 ? y : z;
        const int b = band[o];
        const int lo = b & 0xffff, hi = min(b >> 16, in_n);
        T v = T(0);
        const bool live = (axis == 0 || x < in_n) && (axis == 1 || y < in_n) && (axis == 2 || z < in_n);
        if (live) {
            const int st = axis == 0 ? 1 : axis == 1 ? in_n : in_n * in_n;
            const int base = axis == 0 ? (z * in_n + y) * in_n : axis == 1 ? z * in_n * in_n + x : y * in_n + x;
            // M(o, k) = W[c][o][k] (interpolation) or W[c][k][o] (adjoint)
            const T* wp = Wc + (adjoint ? o : o * n);
            const int wstep = adjoint ? n : 1;
            if (comp) {
                Sum<T> acc;
                for (int k = lo; k < hi; ++k) acc.add(wp[k * wstep], in[base + k * st], true);
                v = acc.get();
            } else {
                T a0 = T(0), a1 = T(0);
                int k = lo;
                for (; k + 1 < hi; k += 2) {
                    a0 = fma(wp[k * wstep], in[base + k * st], a0);
                    a1 = fma(wp[(k + 1) * wstep], in[base + (k + 1) * st], a1);
                }
                if (k < hi) a0 = fma(wp[k * wstep], in[base + k * st], a0);
                v = a0 + a1;
            }
        }
        emit(i, v);
    }
}

// a cube of len values from global memory into shared memory (or scratch)
template <typename T>
__device__ __forceinline__ void stage(T* dst, const T* __restrict__ src, int len) {
    for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = src[i];
}

// shared-memory layout of g_reg / g_interp: W, bands, then (when they fit)
// the two intermediate cubes
template <typename T>
struct RiSmem {
    __host__ __device__ static size_t head(int n) { return (sizeof(T) * 2 * n * n + sizeof(int) * 2 * n + 15) / 16 * 16; }
    __host__ __device__ static size_t cubes(int n) { return sizeof(T) * 2 * size_t(n) * n * n; }
};

// Reg in two launches.  g_reg_xy: a CTA per (parent, child) item takes the
// child's x and y passes (Eq. alg_reg, W_c^T along x then y) into the item's
// slice of the slices buffer (n_parents x 8 cubes of n_I^3).  g_reg_z: a
// thread per parent value sums, children in order, the z passes of the
// present children's slices.
template <typename T>
__global__ void __launch_bounds__(kRiThreads) g_reg_xy(const T* __restrict__ child_src, int child_is_block,
                                                       const int* __restrict__ child_index, int n_parents,
                                                       const T* __restrict__ W, int NI, int comp,
                                                       T* __restrict__ slices, T* __restrict__ scratch,
                                                       int cubes_in_smem) {
    extern __shared__ __align__(16) unsigned char g_smem[];
    const int NB = NI - 1, N3 = NI * NI * NI;
    T* W_s = reinterpret_cast<T*>(g_smem);
    int* band = reinterpret_cast<int*>(W_s + 2 * NI * NI);
    T* t1 = cubes_in_smem ? reinterpret_cast<T*>(g_smem + RiSmem<T>::head(NI))
                          : scratch + int64_t(blockIdx.x) * 2 * N3;
    T* t2 = t1 + N3;
    load_stencil(W_s, band, W, NI, true);
    for (int q = blockIdx.x; q < n_parents * 8; q += gridDim.x) {
        const int s = child_index[q], c = q & 7;
        if (s < 0) continue;                            // uniform over the CTA
        const int cx_ = c & 1, cy_ = (c >> 1) & 1;
        const int in_n = child_is_block ? NB : NI;
        stage(t2, child_is_block ? child_src + int64_t(s) * NB * NB * NB : child_src + int64_t(s) * N3,
              in_n * in_n * in_n);
        __syncthreads();
        pass(t2, in_n, NI, 0, W_s + cx_ * NI * NI, band + cx_ * NI, true, comp != 0, [&](int i, T v) { t1[i] = v; });
        __syncthreads();
        T* out = slices + int64_t(q) * N3;
        pass(t1, NI, NI, 1, W_s + cy_ * NI * NI, band + cy_ * NI, true, comp != 0, [&](int i, T v) { out[i] = v; });
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) g_reg_z(const int* __restrict__ child_index,
                                                    const int* __restrict__ parent_slot, int n_parents,
                                                    T* __restrict__ dst, const T* __restrict__ W, int NI, int comp,
                                                    const T* __restrict__ slices) {
    extern __shared__ __align__(16) unsigned char g_smem[];
    const int N3 = NI * NI * NI;
    T* W_s = reinterpret_cast<T*>(g_smem);
    int* band = reinterpret_cast<int*>(W_s + 2 * NI * NI);
    load_stencil(W_s, band, W, NI, true);
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(n_parents) * N3) return;
    const int p = int(i / N3), e = int(i % N3);
    const int xy = e % (NI * NI), z = e / (NI * NI);
    Sum<T> acc;
    for (int c = 0; c < 8; ++c) {
        if (child_index[int64_t(p) * 8 + c] < 0) continue;
        const int cz_ = c >> 2;
        const int b = band[cz_ * NI + z];
        const T* Wc = W_s + cz_ * NI * NI;
        const T* in = slices + (int64_t(p) * 8 + c) * N3 + xy;
        for (int k = b & 0xffff; k < (b >> 16); ++k) acc.add(Wc[k * NI + z], in[int64_t(k) * NI * NI], comp != 0);
    }
    dst[int64_t(parent_slot[p]) * N3 + e] = acc.get();
}

template <typename T>
__global__ void __launch_bounds__(kRiThreads) g_interp(const int* __restrict__ slot, const int* __restrict__ parent,
                                                     int n_items, T* __restrict__ u, const T* __restrict__ up,
                                                     const T* __restrict__ W, int NI, int accumulate,
                                                     const int* __restrict__ block, int comp,
                                                     T* __restrict__ scratch, int cubes_in_smem) {
    extern __shared__ __align__(16) unsigned char g_smem[];
    const int NB = NI - 1, N3 = NI * NI * NI;
    T* W_s = reinterpret_cast<T*>(g_smem);
    int* band = reinterpret_cast<int*>(W_s + 2 * NI * NI);
    T* t1 = cubes_in_smem ? reinterpret_cast<T*>(g_smem + RiSmem<T>::head(NI))
                          : scratch + int64_t(blockIdx.x) * 2 * N3;
    T* t2 = t1 + N3;
    load_stencil(W_s, band, W, NI, false);
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int s = slot[it], c = s & 7;
        const int cx_ = c & 1, cy_ = (c >> 1) & 1, cz_ = c >> 2;
        stage(t2, up + int64_t(parent[it]) * N3, N3);
        __syncthreads();
        pass(t2, NI, NI, 0, W_s + cx_ * NI * NI, band + cx_ * NI, false, comp != 0, [&](int i, T v) { t1[i] = v; });
        __syncthreads();
        pass(t1, NI, NI, 1, W_s + cy_ * NI * NI, band + cy_ * NI, false, comp != 0, [&](int i, T v) { t2[i] = v; });
        __syncthreads();
        if (block) {
            T* o = u + int64_t(block[it]) * NB * NB * NB;
            pass(t2, NI, NI, 2, W_s + cz_ * NI * NI, band + cz_ * NI, false, comp != 0, [&](int i, T v) {
                const int x = i % NI, y = (i / NI) % NI, z = i / (NI * NI);
                if (x < NB && y < NB && z < NB) o[(z * NB + y) * NB + x] += v;
            });
        } else {
            T* o = u + int64_t(s) * N3;
            pass(t2, NI, NI, 2, W_s + cz_ * NI * NI, band + cz_ * NI, false, comp != 0,
                 [&](int i, T v) { o[i] = accumulate ? o[i] + v : v; });
        }
        __syncthreads();
    }
}

// an item's x-pass outputs in about equal tiles of at most kXTile
inline void x_tiles(int per_item, int* tiles, int* tile_len) {
    *tiles = (per_item + kXTile - 1) / kXTile;
    *tile_len = (per_item + *tiles - 1) / *tiles;
}

inline unsigned grid_for(int64_t total, int threads = kThreads) {
    return unsigned(std::max<int64_t>(1, (total + threads - 1) / threads));
}

// one complex-axis pass (see g_axis); FP64 lines use half the threads per CTA
// so that a CTA's staged columns stay near 64 KB
template <typename T>
cudaError_t axis_pass(const dev::cx<T>* in, const int* in_slots, int64_t in_ws, dev::cx<T>* out,
                      const int* out_slots, int64_t out_ws, int slot_stride, int n, int S, int nin, int nout,
                      int n_other, int64_t axis_stride, int64_t other_stride, int sign, const dev::cx<T>* tw,
                      cudaStream_t st) {
    const int threads = sizeof(T) == 8 ? kLineThreads / 2 : kLineThreads;
    const size_t smem = sizeof(dev::cx<T>) * (size_t(S) + size_t(nin) * threads);
    cudaError_t e = cudaFuncSetAttribute(g_axis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    const int64_t lines = int64_t(n) * n_other * (S / 2 + 1);
    g_axis<T><<<grid_for(lines, threads), threads, smem, st>>>(in, in_slots, in_ws, out, out_slots, out_ws,
                                                              slot_stride, n, S, nin, nout, n_other, axis_stride,
                                                              other_stride, sign, tw);
    return cudaGetLastError();
}

}  // namespace gen

template <typename T>
cudaError_t Generic<T>::r2c(int S, int n_in, const T* src, int64_t stride, const R2CItem* items, int n, void* spec,
                            void* scratch, const void* twt, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int* slots = reinterpret_cast<const int*>(items) + 1;   // R2CItem::dst, 2 ints apart
    using C = dev::cx<T>;
    const int NX = S / 2 + 1;
    const int64_t nws = nws_of(S);
    auto* A = static_cast<C*>(spec);
    auto* B = static_cast<C*>(scratch);
    const auto* tw = static_cast<const C*>(twt);
    // x: rows (z, y < n_in) into A; y: A -> B (planes z < n_in); z: B -> A
    const int64_t bws = int64_t(n_in) * S * NX;
    int tiles = 0, tile_len = 0;
    gen::x_tiles(n_in * n_in * NX, &tiles, &tile_len);
    const size_t smem_x = sizeof(C) * S + sizeof(T) * size_t((tile_len - 1) / NX + 2) * n_in;
    gen::g_r2c_x<T><<<unsigned(int64_t(n) * tiles), gen::kThreads, smem_x, st>>>(src, stride, items, tiles, tile_len,
                                                                                 A, nws, S, n_in, tw);
    cudaError_t e = gen::axis_pass<T>(A, slots, nws, B, nullptr, bws, 2, n, S, n_in, S, n_in, NX, int64_t(S) * NX,
                                      -1, tw, st);
    if (e == cudaSuccess)
        e = gen::axis_pass<T>(B, nullptr, bws, A, slots, nws, 2, n, S, n_in, S, S, int64_t(S) * NX, NX, -1, tw, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t Generic<T>::c2r(int S, int n_out, const void* spec, const C2RItem* items, int n, void* scratch, T* dst,
                            int64_t ds, const T* add, int add_n, int64_t as, const void* twt, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int* slots = reinterpret_cast<const int*>(items);       // C2RItem::src, 3 ints apart
    using C = dev::cx<T>;
    const int NX = S / 2 + 1;
    const int64_t nws = nws_of(S);
    auto* U = const_cast<C*>(static_cast<const C*>(spec));
    auto* V = static_cast<C*>(scratch);
    const auto* tw = static_cast<const C*>(twt);
    // z: U -> V (planes z < n_out); y: V -> U keeping y < n_out; x: U -> reals
    const int64_t vws = int64_t(n_out) * S * NX;
    cudaError_t e = gen::axis_pass<T>(U, slots, nws, V, nullptr, vws, 3, n, S, S, n_out, S, int64_t(S) * NX, NX, +1,
                                      tw, st);
    if (e == cudaSuccess)
        e = gen::axis_pass<T>(V, nullptr, vws, U, slots, nws, 3, n, S, S, n_out, n_out, NX, int64_t(S) * NX, +1, tw,
                              st);
    if (e != cudaSuccess) return e;
    int tiles = 0, tile_len = 0;
    gen::x_tiles(n_out * n_out * n_out, &tiles, &tile_len);
    const size_t smem_x = sizeof(C) * (S + size_t((tile_len - 1) / n_out + 2) * NX);
    gen::g_c2r_x<T><<<unsigned(int64_t(n) * tiles), gen::kThreads, smem_x, st>>>(U, items, tiles, tile_len, dst, ds,
                                                                                 add, add_n, as, nws, S, n_out, tw);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Generic<T>::mac(const void* fh, const void* kh, void* uh, const int* gnbr, int n_groups, int S,
                            int include_self, cudaStream_t st) {
    if (n_groups == 0) return cudaSuccess;
    const int64_t nw = nw_of(S), nws = nws_of(S);
    const int64_t chunks = (nw + 31) / 32;
    // groups per CTA: all of them when the chunks alone give four CTAs per SM
    // (two resident at a time), else fewer so that the grid keeps that size;
    // a multiple of the 8 warps
    const int64_t want = 4 * 152;
    int gpc = n_groups;
    if (chunks < want) gpc = int(std::max<int64_t>(8, int64_t(n_groups) * chunks / want));
    gpc = (gpc + 7) / 8 * 8;
    dim3 block(32, 8), grid(unsigned((n_groups + gpc - 1) / gpc), unsigned(chunks));
    const size_t smem = sizeof(dev::cx<T>) * 343 * 32;
    cudaError_t e = cudaFuncSetAttribute(gen::g_mac<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    gen::g_mac<T><<<grid, block, smem, st>>>(static_cast<const dev::cx<T>*>(fh), static_cast<const dev::cx<T>*>(kh),
                                             static_cast<dev::cx<T>*>(uh), gnbr, n_groups, gpc, include_self, nw, nws);
    return cudaGetLastError();
}

// Reg / Interp: W and its bands in shared memory, and the two intermediate
// cubes too when they fit (else the CTA's 2 n_I^3 slice of the scratch)
template <typename T>
static size_t ri_smem(int NI, int* cubes_in_smem) {
    const size_t head = gen::RiSmem<T>::head(NI), cubes = gen::RiSmem<T>::cubes(NI);
    *cubes_in_smem = head + cubes <= 200 * 1024 ? 1 : 0;
    return head + (*cubes_in_smem ? cubes : 0);
}

template <typename T>
cudaError_t Generic<T>::reg(int n_b, const T* child_src, int child_is_block, const int* child_index,
                            const int* parent_slot, int n_parents, T* dst, const T* W_dev, int comp, T* scratch,
                            T* slices, int n_ctas, cudaStream_t st) {
    if (n_parents == 0) return cudaSuccess;
    const int NI = n_b + 1;
    int in_smem = 0;
    const size_t smem = ri_smem<T>(NI, &in_smem);
    cudaError_t e = cudaFuncSetAttribute(gen::g_reg_xy<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    const int items = 8 * n_parents;
    gen::g_reg_xy<T><<<in_smem ? items : std::min(items, n_ctas), gen::kRiThreads, smem, st>>>(
        child_src, child_is_block, child_index, n_parents, W_dev, NI, comp, slices, scratch, in_smem);
    const size_t smem_z = gen::RiSmem<T>::head(NI);
    gen::g_reg_z<T><<<gen::grid_for(int64_t(n_parents) * NI * NI * NI), gen::kThreads, smem_z, st>>>(
        child_index, parent_slot, n_parents, dst, W_dev, NI, comp, slices);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Generic<T>::interp(int n_b, const int* slot, const int* parent, int n_items, T* u, const T* up,
                               const T* W_dev, int accumulate, const int* block, int comp, T* scratch, int n_ctas,
                               cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    int in_smem = 0;
    const size_t smem = ri_smem<T>(n_b + 1, &in_smem);
    cudaError_t e = cudaFuncSetAttribute(gen::g_interp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    gen::g_interp<T><<<in_smem ? n_items : std::min(n_items, n_ctas), gen::kRiThreads, smem, st>>>(
        slot, parent, n_items, u, up, W_dev, n_b + 1, accumulate, block, comp, scratch, in_smem);
    return cudaGetLastError();
}

template struct Generic<float>;
template struct Generic<double>;

}  // namespace lgf
