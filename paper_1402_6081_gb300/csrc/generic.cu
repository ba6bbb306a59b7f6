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
//  * Products (Eq. alg_mult): a warp per target sibling group and 32
//    frequencies, the chunk's 343 coefficient rows staged in shared memory
//    from the half table, the 8 x 8 sibling products of each neighbour group
//    in registers (mac_block).
//  * Reg and Interp (Eqs. alg_reg, alg_interp): a CTA per item, the three
//    axis passes through a per-CTA scratch in global memory, dense 1D sums
//    over the stencil matrices; compensated FP32 sums where asked.
#include <algorithm>

#include "kernels_impl.cuh"

namespace lgf {
namespace gen {

using dev::cx;
using dev::czero;
using dev::ldg_cx;

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ cx<T> tw(const cx<T>* __restrict__ t, int m) {
    return ldg_cx(t + m);   // (cos, sin)(2 pi m / S)
}
// a * exp(sign i 2 pi m / S)
template <typename T>
__device__ __forceinline__ cx<T> rot(cx<T> a, cx<T> w, int sign) {
    const T s = sign * w.y;
    return {a.x * w.x - a.y * s, a.x * s + a.y * w.x};
}

// ---- forward transform, x: real rows of the input to the first NX values
template <typename T>
__global__ void __launch_bounds__(kThreads) g_r2c_x(const T* __restrict__ src, int64_t stride,
                                                    const R2CItem* __restrict__ items, int n_items,
                                                    cx<T>* __restrict__ A, int64_t nws, int S, int N,
                                                    const cx<T>* __restrict__ twt) {
    const int NX = S / 2 + 1;
    const int64_t total = int64_t(n_items) * N * N * NX;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int k = int(i % NX);
        const int64_t t = i / NX;
        const int r = int(t % (N * N)), it = int(t / (N * N));
        const R2CItem item = items[it];
        const T* row = src + int64_t(item.src) * stride + int64_t(r) * N;
        cx<T> acc = czero<T>();
        for (int x = 0; x < N; ++x) {
            const T v = __ldg(row + x);
            const cx<T> w = tw(twt, (x * k) % S);
            acc.x = fma(v, w.x, acc.x);
            acc.y = fma(-v, w.y, acc.y);
        }
        const int y = r % N, z = r / N;
        A[int64_t(item.dst) * nws + (int64_t(z) * S + y) * NX + k] = acc;
    }
}

// ---- one complex axis (y: stride NX, planes z < N; z: stride S NX, all y)
// out[j] = sum_{m < nin} in[m] exp(sign i 2 pi j m / S), j < nout.  A side
// with slots addresses item it at slots[it * slot_stride] * its stride (the
// level's spectrum buffer), one without at it * its stride (the transform
// scratch, whose items hold only the planes the other passes use).
template <typename T>
__global__ void __launch_bounds__(kThreads) g_axis(const cx<T>* __restrict__ in, const int* __restrict__ in_slots,
                                                   int64_t in_ws, cx<T>* __restrict__ out,
                                                   const int* __restrict__ out_slots, int64_t out_ws,
                                                   int slot_stride, int n_items, int S, int nin, int nout, int n_other,
                                                   int64_t axis_stride, int64_t other_stride, int sign,
                                                   const cx<T>* __restrict__ twt) {
    // thread (item, other, j, kx): kx fastest
    const int NX = S / 2 + 1;
    const int64_t total = int64_t(n_items) * n_other * nout * NX;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int kx = int(i % NX);
        int64_t t = i / NX;
        const int j = int(t % nout);
        t /= nout;
        const int o = int(t % n_other), it = int(t / n_other);
        const int64_t line = int64_t(o) * other_stride + kx;
        const int64_t ib = (in_slots ? int64_t(in_slots[int64_t(it) * slot_stride]) : int64_t(it)) * in_ws + line;
        const int64_t ob = (out_slots ? int64_t(out_slots[int64_t(it) * slot_stride]) : int64_t(it)) * out_ws + line;
        cx<T> acc = czero<T>();
        for (int m = 0; m < nin; ++m) {
            const cx<T> v = ldg_cx(in + ib + int64_t(m) * axis_stride);
            const cx<T> p = rot(v, tw(twt, (j * m) % S), sign);
            acc.x += p.x;
            acc.y += p.y;
        }
        out[ob + int64_t(j) * axis_stride] = acc;
    }
}

// ---- inverse transform, x: Hermitian rows to the first N real samples (+ add)
template <typename T>
__global__ void __launch_bounds__(kThreads) g_c2r_x(const cx<T>* __restrict__ U, const C2RItem* __restrict__ items,
                                                    int n_items, T* __restrict__ dst, int64_t dst_stride,
                                                    const T* __restrict__ add, int add_n, int64_t add_stride,
                                                    int64_t nws, int S, int N, const cx<T>* __restrict__ twt) {
    const int NX = S / 2 + 1;
    const int64_t total = int64_t(n_items) * N * N * N;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int x = int(i % N);
        const int64_t t = i / N;
        const int r = int(t % (N * N)), it = int(t / (N * N));
        const C2RItem item = items[it];
        const int y = r % N, z = r / N;
        const cx<T>* row = U + int64_t(item.src) * nws + (int64_t(z) * S + y) * NX;
        // x[n] = X[0] + 2 sum_{0 < k < S/2} Re(X[k] e^{+i 2 pi n k / S}) + X[S/2] (-1)^n (S even)
        T acc = ldg_cx(row).x;
        const int kmax = (S % 2 == 0) ? S / 2 : NX;
        for (int k = 1; k < kmax; ++k) {
            const cx<T> v = ldg_cx(row + k), w = tw(twt, (x * k) % S);
            acc += T(2) * (v.x * w.x - v.y * w.y);
        }
        if (S % 2 == 0) acc += ((x & 1) ? T(-1) : T(1)) * ldg_cx(row + S / 2).x;
        if (add != nullptr && item.aux >= 0) acc += __ldg(add + int64_t(item.aux) * add_stride + (int64_t(z) * add_n + y) * add_n + x);
        dst[int64_t(item.dst) * dst_stride + int64_t(r) * N + x] = acc;
    }
}

// ---- products
template <typename T>
__global__ void __launch_bounds__(256) g_mac(const cx<T>* __restrict__ fh, const cx<T>* __restrict__ kh,
                                             cx<T>* __restrict__ uh, const int* __restrict__ gnbr, int n_groups,
                                             int include_self, int64_t nw, int64_t nws) {
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
    const int g = blockIdx.x * 8 + threadIdx.y;
    const int64_t w = w0 + threadIdx.x;
    if (g >= n_groups) return;
    const int64_t wc = w < nw ? w : nw - 1;
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

// ---- Reg and Interp: one 1D pass over a cube, out[..] (+)= sum_k M(i, k) in[..]
// with M(i, k) = W[c][i][k] (interpolation) or W[c][k][i] (its adjoint)
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

// axis a of a cube of edge n (stride 1, n, n^2): out[i along a] = sum_k M(i, k) in[k along a]
template <typename T>
__device__ void pass(const T* __restrict__ in, int in_n, T* __restrict__ out, int n, int axis,
                     const T* __restrict__ Wc, bool adjoint, bool comp, bool accumulate) {
    const int n3 = n * n * n;
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int x = i % n, y = (i / n) % n, z = i / (n * n);
        const int o = axis == 0 ? x : axis == 1 ? y : z;
        Sum<T> acc;
        for (int k = 0; k < in_n; ++k) {
            const T w = adjoint ? Wc[k * n + o] : Wc[o * n + k];
            if (w == T(0)) continue;
            const int xi = axis == 0 ? k : x, yi = axis == 1 ? k : y, zi = axis == 2 ? k : z;
            if (xi >= in_n || yi >= in_n || zi >= in_n) continue;
            acc.add(w, in[(zi * in_n + yi) * in_n + xi], comp);
        }
        if (accumulate) out[i] += acc.get();
        else out[i] = acc.get();
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) g_reg(const T* __restrict__ child_src, int child_is_block,
                                                  const int* __restrict__ child_index,
                                                  const int* __restrict__ parent_slot, int n_parents,
                                                  T* __restrict__ dst, const T* __restrict__ W, int NI, int comp,
                                                  T* __restrict__ scratch) {
    const int NB = NI - 1, N3 = NI * NI * NI;
    T* t1 = scratch + int64_t(blockIdx.x) * 3 * N3;
    T* t2 = t1 + N3;
    T* tc = t2 + N3;   // a block child padded to NI^3
    for (int p = blockIdx.x; p < n_parents; p += gridDim.x) {
        T* out = dst + int64_t(parent_slot[p]) * N3;
        for (int i = threadIdx.x; i < N3; i += blockDim.x) out[i] = T(0);
        __syncthreads();
        for (int c = 0; c < 8; ++c) {
            const int s = child_index[int64_t(p) * 8 + c];
            if (s < 0) continue;
            const T* in;
            if (child_is_block) {
                const T* b = child_src + int64_t(s) * NB * NB * NB;
                for (int i = threadIdx.x; i < N3; i += blockDim.x) {
                    const int x = i % NI, y = (i / NI) % NI, z = i / (NI * NI);
                    tc[i] = (x < NB && y < NB && z < NB) ? b[(z * NB + y) * NB + x] : T(0);
                }
                __syncthreads();
                in = tc;
            } else {
                in = child_src + int64_t(s) * N3;
            }
            const int cx_ = c & 1, cy_ = (c >> 1) & 1, cz_ = c >> 2;
            pass(in, NI, t1, NI, 0, W + int64_t(cx_) * NI * NI, true, comp != 0, false);
            __syncthreads();
            pass(t1, NI, t2, NI, 1, W + int64_t(cy_) * NI * NI, true, comp != 0, false);
            __syncthreads();
            pass(t2, NI, out, NI, 2, W + int64_t(cz_) * NI * NI, true, comp != 0, true);
            __syncthreads();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) g_interp(const int* __restrict__ slot, const int* __restrict__ parent,
                                                     int n_items, T* __restrict__ u, const T* __restrict__ up,
                                                     const T* __restrict__ W, int NI, int accumulate,
                                                     const int* __restrict__ block, int comp,
                                                     T* __restrict__ scratch) {
    const int NB = NI - 1, N3 = NI * NI * NI;
    T* t1 = scratch + int64_t(blockIdx.x) * 3 * N3;
    T* t2 = t1 + N3;
    T* t3 = t2 + N3;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int s = slot[it], c = s & 7;
        const T* U = up + int64_t(parent[it]) * N3;
        pass(U, NI, t1, NI, 0, W + int64_t(c & 1) * NI * NI, false, comp != 0, false);
        __syncthreads();
        pass(t1, NI, t2, NI, 1, W + int64_t((c >> 1) & 1) * NI * NI, false, comp != 0, false);
        __syncthreads();
        pass(t2, NI, t3, NI, 2, W + int64_t(c >> 2) * NI * NI, false, comp != 0, false);
        __syncthreads();
        if (block) {
            T* o = u + int64_t(block[it]) * NB * NB * NB;
            for (int i = threadIdx.x; i < NB * NB * NB; i += blockDim.x) {
                const int x = i % NB, y = (i / NB) % NB, z = i / (NB * NB);
                o[i] += t3[(z * NI + y) * NI + x];
            }
        } else {
            T* o = u + int64_t(s) * N3;
            for (int i = threadIdx.x; i < N3; i += blockDim.x) o[i] = accumulate ? o[i] + t3[i] : t3[i];
        }
        __syncthreads();
    }
}

inline unsigned grid_for(int64_t total) {
    return unsigned(std::max<int64_t>(1, std::min<int64_t>((total + kThreads - 1) / kThreads, 152 * 32)));
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
    gen::g_r2c_x<T><<<gen::grid_for(int64_t(n) * n_in * n_in * NX), gen::kThreads, 0, st>>>(
        src, stride, items, n, A, nws, S, n_in, tw);
    gen::g_axis<T><<<gen::grid_for(int64_t(n) * n_in * S * NX), gen::kThreads, 0, st>>>(
        A, slots, nws, B, nullptr, bws, 2, n, S, n_in, S, n_in, NX, int64_t(S) * NX, -1, tw);
    gen::g_axis<T><<<gen::grid_for(int64_t(n) * S * S * NX), gen::kThreads, 0, st>>>(
        B, nullptr, bws, A, slots, nws, 2, n, S, n_in, S, S, int64_t(S) * NX, NX, -1, tw);
    return cudaGetLastError();
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
    gen::g_axis<T><<<gen::grid_for(int64_t(n) * S * n_out * NX), gen::kThreads, 0, st>>>(
        U, slots, nws, V, nullptr, vws, 3, n, S, S, n_out, S, int64_t(S) * NX, NX, +1, tw);
    gen::g_axis<T><<<gen::grid_for(int64_t(n) * n_out * n_out * NX), gen::kThreads, 0, st>>>(
        V, nullptr, vws, U, slots, nws, 3, n, S, S, n_out, n_out, NX, int64_t(S) * NX, +1, tw);
    gen::g_c2r_x<T><<<gen::grid_for(int64_t(n) * n_out * n_out * n_out), gen::kThreads, 0, st>>>(
        U, items, n, dst, ds, add, add_n, as, nws, S, n_out, tw);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Generic<T>::mac(const void* fh, const void* kh, void* uh, const int* gnbr, int n_groups, int S,
                            int include_self, cudaStream_t st) {
    if (n_groups == 0) return cudaSuccess;
    const int64_t nw = nw_of(S), nws = nws_of(S);
    dim3 block(32, 8), grid((n_groups + 7) / 8, unsigned((nw + 31) / 32));
    const size_t smem = sizeof(dev::cx<T>) * 343 * 32;
    cudaError_t e = cudaFuncSetAttribute(gen::g_mac<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    gen::g_mac<T><<<grid, block, smem, st>>>(static_cast<const dev::cx<T>*>(fh), static_cast<const dev::cx<T>*>(kh),
                                             static_cast<dev::cx<T>*>(uh), gnbr, n_groups, include_self, nw, nws);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Generic<T>::reg(int n_b, const T* child_src, int child_is_block, const int* child_index,
                            const int* parent_slot, int n_parents, T* dst, const T* W_dev, int comp, T* scratch,
                            int n_ctas, cudaStream_t st) {
    if (n_parents == 0) return cudaSuccess;
    gen::g_reg<T><<<std::min(n_parents, n_ctas), gen::kThreads, 0, st>>>(
        child_src, child_is_block, child_index, parent_slot, n_parents, dst, W_dev, n_b + 1, comp, scratch);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Generic<T>::interp(int n_b, const int* slot, const int* parent, int n_items, T* u, const T* up,
                               const T* W_dev, int accumulate, const int* block, int comp, T* scratch, int n_ctas,
                               cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    gen::g_interp<T><<<std::min(n_items, n_ctas), gen::kThreads, 0, st>>>(
        slot, parent, n_items, u, up, W_dev, n_b + 1, accumulate, block, comp, scratch);
    return cudaGetLastError();
}

template struct Generic<float>;
template struct Generic<double>;

}  // namespace lgf
