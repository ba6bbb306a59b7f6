// Device kernels of one FLGF solve (Sec. 3.1 Steps 1-3), templated on the
// arithmetic type T (float or double).  Included by kernels_f32.cu and
// kernels_f64.cu, which instantiate the launchers.
//
// Spectrum layout: one block/interval spectrum is NW = NX*S*S complex values,
// w = (kz*S + ky)*NX + kx with NX = S/2 + 1 (R2C along x).  Spectra of a level
// live in "slots": slot = group*8 + child, where a group is a 2x2x2 set of
// siblings (interval index >> 1) and child = cx + 2cy + 4cz; absent siblings
// keep an all-zero slot so the interaction kernels need no per-source test.
#pragma once

#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "lgf_internal.h"

namespace lgf {
namespace dev {

template <typename T>
__device__ __forceinline__ cx<T> ldg_cx(const cx<T>* p) {
    cx<T> v;
    v.x = __ldg(&p->x);
    v.y = __ldg(&p->y);
    return v;
}
template <>
__device__ __forceinline__ cx<float> ldg_cx<float>(const cx<float>* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
template <>
__device__ __forceinline__ cx<double> ldg_cx<double>(const cx<double>* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}

constexpr int kFftThreads = 256;

// ---------------------------------------------------------------------------
// Padded R2C (Eq. alg_upfft): an NIN^3 real cube, zero-padded to S^3, to its
// half spectrum.  One CTA per item; the partially transformed cube stays in
// shared memory as B[(z*S + ky)*NX + kx], z < NIN (only NIN z-planes are
// non-zero until the last pass, which goes straight to global memory).
template <typename T, int S, int NIN>
__global__ void __launch_bounds__(kFftThreads) k_r2c(const T* __restrict__ src, int64_t src_stride,
                                                     const R2CItem* __restrict__ items,
                                                     cx<T>* __restrict__ spec) {
    constexpr int NX = S / 2 + 1;
    constexpr int64_t NW = int64_t(NX) * S * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* B = reinterpret_cast<cx<T>*>(smem_raw);
    const R2CItem it = items[blockIdx.x];
    const T* in = src + int64_t(it.src) * src_stride;
    cx<T>* out = spec + int64_t(it.dst) * NW;

    // x pass: two real lines per complex transform
    constexpr int NL = NIN * NIN, NP = (NL + 1) / 2;
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        const int l0 = 2 * p, l1 = 2 * p + 1;
        const bool has1 = l1 < NL;
        const T* r0 = in + int64_t(l0) * NIN;
        const T* r1 = in + int64_t(has1 ? l1 : l0) * NIN;
        cx<T> z[S];
#pragma unroll
        for (int x = 0; x < S; ++x)
            z[x] = x < NIN ? cx<T>{r0[x], has1 ? r1[x] : T(0)} : czero<T>();
        fft<S, S, -1, NIN>(z);
        const int y0 = l0 % NIN, z0 = l0 / NIN, y1 = l1 % NIN, z1 = l1 / NIN;
        cx<T>* d0 = B + (z0 * S + y0) * NX;
        cx<T>* d1 = B + (z1 * S + y1) * NX;
#pragma unroll
        for (int k = 0; k < NX; ++k) {
            const cx<T> a = z[k], b = z[(S - k) % S];
            d0[k] = {T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y)};
            if (has1) d1[k] = {T(0.5) * (a.y + b.y), T(0.5) * (b.x - a.x)};
        }
    }
    __syncthreads();
    // y pass: lines (kx, z), in place within the column
    for (int l = threadIdx.x; l < NX * NIN; l += blockDim.x) {
        const int kx = l % NX, zz = l / NX;
        cx<T>* col = B + zz * S * NX + kx;
        cx<T> v[S];
#pragma unroll
        for (int y = 0; y < S; ++y) v[y] = y < NIN ? col[y * NX] : czero<T>();
        fft<S, S, -1, NIN>(v);
#pragma unroll
        for (int y = 0; y < S; ++y) col[y * NX] = v[y];
    }
    __syncthreads();
    // z pass: lines (kx, ky), results to global (coalesced across the CTA)
    for (int l = threadIdx.x; l < NX * S; l += blockDim.x) {
        const cx<T>* col = B + l;
        cx<T> v[S];
#pragma unroll
        for (int zz = 0; zz < S; ++zz) v[zz] = zz < NIN ? col[zz * S * NX] : czero<T>();
        fft<S, S, -1, NIN>(v);
#pragma unroll
        for (int kz = 0; kz < S; ++kz) out[int64_t(kz) * S * NX + l] = v[kz];
    }
}

// ---------------------------------------------------------------------------
// Truncated C2R (Eq. alg_dwfft): keep the first NOUT samples per axis.
//   dst[item.dst*dst_stride + (z*NOUT + y)*NOUT + x] = v (+ add[item.aux*add_stride
//   + (z*add_n + y)*add_n + x] when add != null and item.aux >= 0)
// The 1/S^3 of the inverse transform is folded into the kernel spectra.
template <typename T, int S, int NOUT>
__global__ void __launch_bounds__(kFftThreads) k_c2r(const cx<T>* __restrict__ spec,
                                                     const C2RItem* __restrict__ items,
                                                     T* __restrict__ dst, int64_t dst_stride,
                                                     const T* __restrict__ add, int add_n,
                                                     int64_t add_stride) {
    constexpr int NX = S / 2 + 1;
    constexpr int64_t NW = int64_t(NX) * S * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* B = reinterpret_cast<cx<T>*>(smem_raw);
    const C2RItem it = items[blockIdx.x];
    const cx<T>* in = spec + int64_t(it.src) * NW;

    // z pass: lines (kx, ky); keep z < NOUT
    for (int l = threadIdx.x; l < NX * S; l += blockDim.x) {
        cx<T> v[S];
#pragma unroll
        for (int kz = 0; kz < S; ++kz) v[kz] = ldg_cx(in + int64_t(kz) * S * NX + l);
        fft<S, S, 1, S>(v);
#pragma unroll
        for (int zz = 0; zz < NOUT; ++zz) B[zz * S * NX + l] = v[zz];
    }
    __syncthreads();
    // y pass: lines (kx, z < NOUT); keep y < NOUT
    for (int l = threadIdx.x; l < NX * NOUT; l += blockDim.x) {
        const int kx = l % NX, zz = l / NX;
        cx<T>* col = B + zz * S * NX + kx;
        cx<T> v[S];
#pragma unroll
        for (int y = 0; y < S; ++y) v[y] = col[y * NX];
        fft<S, S, 1, S>(v);
#pragma unroll
        for (int y = 0; y < NOUT; ++y) col[y * NX] = v[y];
    }
    __syncthreads();
    // x pass: two Hermitian half-lines per complex inverse transform
    constexpr int NL = NOUT * NOUT, NP = (NL + 1) / 2;
    T* out = dst + int64_t(it.dst) * dst_stride;
    const T* ad = (add != nullptr && it.aux >= 0) ? add + int64_t(it.aux) * add_stride : nullptr;
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        const int l0 = 2 * p, l1 = 2 * p + 1;
        const bool has1 = l1 < NL;
        const int y0 = l0 % NOUT, z0 = l0 / NOUT, y1 = l1 % NOUT, z1 = l1 / NOUT;
        const cx<T>* a = B + (z0 * S + y0) * NX;
        const cx<T>* b = B + ((has1 ? z1 : z0) * S + (has1 ? y1 : y0)) * NX;
        cx<T> z[S];
#pragma unroll
        for (int k = 0; k < NX; ++k) {
            cx<T> A = a[k], Bk = has1 ? b[k] : czero<T>();
            if (k == 0 || 2 * k == S) {   // exactly real for a real signal
                A.y = T(0);
                Bk.y = T(0);
            }
            z[k] = {A.x - Bk.y, A.y + Bk.x};
            if (k > 0 && S - k >= NX) z[S - k] = {A.x + Bk.y, Bk.x - A.y};
        }
        fft<S, S, 1, S>(z);
        T* o0 = out + (z0 * NOUT + y0) * NOUT;
        T* o1 = out + (z1 * NOUT + y1) * NOUT;
        const T* a0 = ad ? ad + (z0 * add_n + y0) * add_n : nullptr;
        const T* a1 = ad ? ad + (z1 * add_n + y1) * add_n : nullptr;
#pragma unroll
        for (int x = 0; x < NOUT; ++x) {
            o0[x] = a0 ? z[x].x + a0[x] : z[x].x;
            if (has1) o1[x] = a1 ? z[x].y + a1[x] : z[x].y;
        }
    }
}

// ---------------------------------------------------------------------------
// Level-0 near-field products (Eq. alg_mult with InflList = near neighbours):
//   uh[P] = sum_{Q near P} fh[Q] * k0^{Q-P},  per frequency w.
// Thread = (w, one sibling group g of 8 target blocks).  The 27 kernel
// coefficients of w sit in registers; the 64 source blocks around the group
// (4^3) are each loaded once and applied to every target within reach (216
// products).  Block-dim (32, G): the 32 lanes of a warp take 32 consecutive
// w of one group, so every load is one coalesced 256 B (FP32) line.
template <typename T>
__global__ void __launch_bounds__(256) k_mac_level0(const cx<T>* __restrict__ fh,
                                                    const cx<T>* __restrict__ kh,
                                                    cx<T>* __restrict__ uh,
                                                    const int* __restrict__ gnbr, int n_groups,
                                                    int64_t NW) {
    const int64_t w = int64_t(blockIdx.y) * 32 + threadIdx.x;
    const int g = blockIdx.x * blockDim.y + threadIdx.y;
    if (g >= n_groups || w >= NW) return;
    cx<T> k[27];
#pragma unroll
    for (int d = 0; d < 27; ++d) k[d] = ldg_cx(kh + int64_t(d) * NW + w);
    cx<T> acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = czero<T>();
    const int* nb = gnbr + int64_t(g) * 27;
#pragma unroll
    for (int tz = -1; tz <= 2; ++tz)
#pragma unroll
        for (int ty = -1; ty <= 2; ++ty)
#pragma unroll
            for (int tx = -1; tx <= 2; ++tx) {
                const int ex = tx < 0 ? -1 : tx >> 1, ey = ty < 0 ? -1 : ty >> 1,
                          ez = tz < 0 ? -1 : tz >> 1;
                const int q = __ldg(nb + (ex + 1) + 3 * (ey + 1) + 9 * (ez + 1));
                if (q < 0) continue;
                const int cs = (tx - 2 * ex) + 2 * (ty - 2 * ey) + 4 * (tz - 2 * ez);
                const cx<T> F = ldg_cx(fh + (int64_t(q) * 8 + cs) * NW + w);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int dx = tx - (c & 1), dy = ty - ((c >> 1) & 1), dz = tz - (c >> 2);
                    if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) continue;
                    acc[c] = cmac(acc[c], F, k[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)]);
                }
            }
#pragma unroll
    for (int c = 0; c < 8; ++c) uh[(int64_t(g) * 8 + c) * NW + w] = acc[c];
}

// ---------------------------------------------------------------------------
// Level >= 1 interaction-list products (Eq. alg_mult with the interaction list):
//   uh[P] = sum_{Q in IL(P)} fh[Q] * k^{Q-P},  per frequency w.
// Every interval Q of IL(P) is a child of one of the 26 neighbour groups
// g+e of P's sibling group g.  Thread = (w, group g): for each e it loads the
// 8 source spectra of group g+e and the 27 coefficients k^{2e+delta}, delta
// in [-1,1]^3, and applies all 8x8 (target, source) products, the offset
// being d = 2e + c_src - c_tgt.  The coefficient table holds all 7^3 offsets
// with zeros at the 27 near ones (|d| <= 1), which removes the list test.
// The CTA stages the coefficients of its 32 frequencies in shared memory
// (343 x 32), shared by its G groups.
template <typename T>
__global__ void __launch_bounds__(256) k_mac_interval(const cx<T>* __restrict__ fh,
                                                      const cx<T>* __restrict__ kh,
                                                      cx<T>* __restrict__ uh,
                                                      const int* __restrict__ gnbr, int n_groups,
                                                      int64_t NW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* sk = reinterpret_cast<cx<T>*>(smem_raw);   // [343][32]
    const int64_t w0 = int64_t(blockIdx.y) * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    for (int i = tid; i < 343 * 32; i += nthr) {
        const int d = i >> 5, lane = i & 31;
        const int64_t w = w0 + lane;
        sk[i] = w < NW ? ldg_cx(kh + int64_t(d) * NW + w) : czero<T>();
    }
    __syncthreads();
    const int g = blockIdx.x * blockDim.y + threadIdx.y;
    if (g >= n_groups) return;
    const int64_t w = w0 + threadIdx.x;
    const int64_t wc = w < NW ? w : NW - 1;
    cx<T> acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = czero<T>();
    const int* nb = gnbr + int64_t(g) * 27;
#pragma unroll 1
    for (int e = 0; e < 27; ++e) {
        if (e == 13) continue;
        const int q = __ldg(nb + e);
        if (q < 0) continue;
        const int ex = e % 3 - 1, ey = (e / 3) % 3 - 1, ez = e / 9 - 1;
        cx<T> F[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) F[c] = ldg_cx(fh + (int64_t(q) * 8 + c) * NW + wc);
        const cx<T>* kb = sk + ((2 * ex + 3) + 7 * (2 * ey + 3) + 49 * (2 * ez + 3)) * 32 + threadIdx.x;
        cx<T> kk[27];
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx)
                    kk[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] = kb[(dx + 7 * dy + 49 * dz) * 32];
#pragma unroll
        for (int ct = 0; ct < 8; ++ct)
#pragma unroll
            for (int cs = 0; cs < 8; ++cs) {
                const int dx = (cs & 1) - (ct & 1), dy = ((cs >> 1) & 1) - ((ct >> 1) & 1),
                          dz = (cs >> 2) - (ct >> 2);
                acc[ct] = cmac(acc[ct], F[cs], kk[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)]);
            }
    }
    if (w < NW) {
#pragma unroll
        for (int c = 0; c < 8; ++c) uh[(int64_t(g) * 8 + c) * NW + w] = acc[c];
    }
}

// ---------------------------------------------------------------------------
// Reg (Eq. alg_reg): parent sources = sum over the 8 children c of
// (W_cz^T x W_cy^T x W_cx^T) child sources.  One CTA per parent interval;
// W[c][i][p] is the weight of parent node p for child node i.  A level-1 child
// is a block: its sources occupy nodes [0, n_b)^3 and its last node plane is 0.
template <typename T>
__global__ void k_reg(int n_b, const T* __restrict__ child_src, int child_is_block,
                      const int* __restrict__ child_index, const int* __restrict__ parent_slot,
                      T* __restrict__ dst, const T* __restrict__ W) {
    const int nI = n_b + 1, N3 = nI * nI * nI;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ws = reinterpret_cast<T*>(smem_raw);   // [2][nI][nI]
    T* in = Ws + 2 * nI * nI;
    T* t1 = in + N3;
    T* acc = t1 + N3;
    for (int i = threadIdx.x; i < 2 * nI * nI; i += blockDim.x) Ws[i] = W[i];
    for (int i = threadIdx.x; i < N3; i += blockDim.x) acc[i] = T(0);
    for (int c = 0; c < 8; ++c) {
        const int src = child_index[blockIdx.x * 8 + c];
        if (src < 0) continue;
        const int cxp = c & 1, cyp = (c >> 1) & 1, czp = c >> 2;
        __syncthreads();
        for (int i = threadIdx.x; i < N3; i += blockDim.x) {
            const int x = i % nI, y = (i / nI) % nI, z = i / (nI * nI);
            T v;
            if (child_is_block)
                v = (x < n_b && y < n_b && z < n_b)
                        ? child_src[int64_t(src) * n_b * n_b * n_b + (z * n_b + y) * n_b + x]
                        : T(0);
            else
                v = child_src[int64_t(src) * N3 + i];
            in[i] = v;
        }
        __syncthreads();
        const T* Wx = Ws + cxp * nI * nI;
        const T* Wy = Ws + cyp * nI * nI;
        const T* Wz = Ws + czp * nI * nI;
        // x: t1[z][y][p] = sum_i Wx[i][p] in[z][y][i]
        for (int i = threadIdx.x; i < N3; i += blockDim.x) {
            const int p = i % nI, zy = i / nI;
            T s = T(0);
            for (int k = 0; k < nI; ++k) s = fma(Wx[k * nI + p], in[zy * nI + k], s);
            t1[i] = s;
        }
        __syncthreads();
        // y: in[z][q][p] = sum_j Wy[j][q] t1[z][j][p]
        for (int i = threadIdx.x; i < N3; i += blockDim.x) {
            const int p = i % nI, q = (i / nI) % nI, z = i / (nI * nI);
            T s = T(0);
            for (int k = 0; k < nI; ++k) s = fma(Wy[k * nI + q], t1[(z * nI + k) * nI + p], s);
            in[i] = s;
        }
        __syncthreads();
        // z: acc[r][q][p] += sum_k Wz[k][r] in[k][q][p]
        for (int i = threadIdx.x; i < N3; i += blockDim.x) {
            const int qp = i % (nI * nI), r = i / (nI * nI);
            T s = acc[i];
            for (int k = 0; k < nI; ++k) s = fma(Wz[k * nI + r], in[k * nI * nI + qp], s);
            acc[i] = s;
        }
    }
    __syncthreads();
    T* out = dst + int64_t(parent_slot[blockIdx.x]) * N3;
    for (int i = threadIdx.x; i < N3; i += blockDim.x) out[i] = acc[i];
}

// ---------------------------------------------------------------------------
// Interp (Eq. alg_interp): u[slot] += (W_cz x W_cy x W_cx) up[parent] with
// c = slot & 7 the interval's position among its siblings.
template <typename T>
__global__ void k_interp(int n_b, const int* __restrict__ slot, const int* __restrict__ parent,
                         T* __restrict__ u, const T* __restrict__ up, const T* __restrict__ W) {
    const int nI = n_b + 1, N3 = nI * nI * nI;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ws = reinterpret_cast<T*>(smem_raw);
    T* a = Ws + 2 * nI * nI;
    T* b = a + N3;
    const int s = slot[blockIdx.x];
    const int c = s & 7, cxp = c & 1, cyp = (c >> 1) & 1, czp = c >> 2;
    for (int i = threadIdx.x; i < 2 * nI * nI; i += blockDim.x) Ws[i] = W[i];
    const T* U = up + int64_t(parent[blockIdx.x]) * N3;
    for (int i = threadIdx.x; i < N3; i += blockDim.x) a[i] = U[i];
    __syncthreads();
    const T* Wx = Ws + cxp * nI * nI;
    const T* Wy = Ws + cyp * nI * nI;
    const T* Wz = Ws + czp * nI * nI;
    // x: b[pz][py][ix] = sum_px Wx[ix][px] a[pz][py][px]
    for (int i = threadIdx.x; i < N3; i += blockDim.x) {
        const int ix = i % nI, zy = i / nI;
        T acc = T(0);
        for (int k = 0; k < nI; ++k) acc = fma(Wx[ix * nI + k], a[zy * nI + k], acc);
        b[i] = acc;
    }
    __syncthreads();
    // y: a[pz][iy][ix] = sum_py Wy[iy][py] b[pz][py][ix]
    for (int i = threadIdx.x; i < N3; i += blockDim.x) {
        const int ix = i % nI, iy = (i / nI) % nI, z = i / (nI * nI);
        T acc = T(0);
        for (int k = 0; k < nI; ++k) acc = fma(Wy[iy * nI + k], b[(z * nI + k) * nI + ix], acc);
        a[i] = acc;
    }
    __syncthreads();
    // z: u[iz][iy][ix] += sum_pz Wz[iz][pz] a[pz][iy][ix]
    T* out = u + int64_t(s) * N3;
    for (int i = threadIdx.x; i < N3; i += blockDim.x) {
        const int yx = i % (nI * nI), iz = i / (nI * nI);
        T acc = T(0);
        for (int k = 0; k < nI; ++k) acc = fma(Wz[iz * nI + k], a[k * nI * nI + yx], acc);
        out[i] += acc;
    }
}

}  // namespace dev

// ---------------------------------------------------------------------------
// Launchers

template <typename T, int S, int NIN>
static cudaError_t launch_r2c(const T* src, int64_t stride, const R2CItem* items, int n,
                              void* spec, cudaStream_t st) {
    constexpr int NX = S / 2 + 1;
    const size_t smem = sizeof(dev::cx<T>) * NIN * S * NX;
    auto k = dev::k_r2c<T, S, NIN>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    k<<<n, dev::kFftThreads, smem, st>>>(src, stride, items, static_cast<dev::cx<T>*>(spec));
    return cudaGetLastError();
}

template <typename T, int S, int NOUT>
static cudaError_t launch_c2r(const void* spec, const C2RItem* items, int n, T* dst, int64_t ds,
                              const T* add, int add_n, int64_t as, cudaStream_t st) {
    constexpr int NX = S / 2 + 1;
    const size_t smem = sizeof(dev::cx<T>) * NOUT * S * NX;
    auto k = dev::k_c2r<T, S, NOUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    k<<<n, dev::kFftThreads, smem, st>>>(static_cast<const dev::cx<T>*>(spec), items, dst, ds, add,
                                         add_n, as);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::r2c(int S, int n_in, const T* src, int64_t stride, const R2CItem* items,
                           int n, void* spec, cudaStream_t st) {
#define LGF_R2C(SS, NN) \
    if (S == SS && n_in == NN) return launch_r2c<T, SS, NN>(src, stride, items, n, spec, st);
    LGF_R2C(8, 4) LGF_R2C(10, 4) LGF_R2C(10, 5)
    LGF_R2C(16, 8) LGF_R2C(17, 8) LGF_R2C(17, 9) LGF_R2C(18, 8) LGF_R2C(18, 9)
    LGF_R2C(32, 16) LGF_R2C(33, 16) LGF_R2C(33, 17) LGF_R2C(34, 16) LGF_R2C(34, 17)
    LGF_R2C(36, 16) LGF_R2C(36, 17)
#undef LGF_R2C
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::c2r(int S, int n_out, const void* spec, const C2RItem* items, int n, T* dst,
                           int64_t ds, const T* add, int add_n, int64_t as, cudaStream_t st) {
#define LGF_C2R(SS, NN) \
    if (S == SS && n_out == NN) return launch_c2r<T, SS, NN>(spec, items, n, dst, ds, add, add_n, as, st);
    LGF_C2R(8, 4) LGF_C2R(10, 5)
    LGF_C2R(16, 8) LGF_C2R(17, 9) LGF_C2R(18, 9)
    LGF_C2R(32, 16) LGF_C2R(33, 17) LGF_C2R(34, 17) LGF_C2R(36, 17)
#undef LGF_C2R
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::mac_level0(const void* fh, const void* kh, void* uh, const int* gnbr,
                                  int n_groups, int S, cudaStream_t st) {
    if (n_groups == 0) return cudaSuccess;
    const int64_t NW = nw_of(S);
    const int G = 8;
    dim3 block(32, G), grid((n_groups + G - 1) / G, unsigned((NW + 31) / 32));
    dev::k_mac_level0<T><<<grid, block, 0, st>>>(static_cast<const dev::cx<T>*>(fh),
                                                 static_cast<const dev::cx<T>*>(kh),
                                                 static_cast<dev::cx<T>*>(uh), gnbr, n_groups, NW);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::mac_interval(const void* fh, const void* kh, void* uh, const int* gnbr,
                                    int n_groups, int S, cudaStream_t st) {
    const size_t smem = sizeof(dev::cx<T>) * 343 * 32;
    auto k = dev::k_mac_interval<T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    if (n_groups == 0) return cudaSuccess;
    const int64_t NW = nw_of(S);
    const int G = 8;
    dim3 block(32, G), grid((n_groups + G - 1) / G, unsigned((NW + 31) / 32));
    k<<<grid, block, smem, st>>>(static_cast<const dev::cx<T>*>(fh),
                                 static_cast<const dev::cx<T>*>(kh),
                                 static_cast<dev::cx<T>*>(uh), gnbr, n_groups, NW);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::reg(int n_b, int /*n_max*/, const T* child_src, int child_is_block,
                           const int* child_index, const int* parent_slot, int n_parents, T* dst,
                           const T* W, cudaStream_t st) {
    if (n_parents == 0) return cudaSuccess;
    const int nI = n_b + 1;
    const size_t smem = sizeof(T) * (2 * nI * nI + 3 * nI * nI * nI);
    auto k = dev::k_reg<T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k<<<n_parents, 256, smem, st>>>(n_b, child_src, child_is_block, child_index, parent_slot, dst, W);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::interp(int n_b, const int* slot, const int* parent, int n_items, T* u,
                              const T* up, const T* W, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const int nI = n_b + 1;
    const size_t smem = sizeof(T) * (2 * nI * nI + 2 * nI * nI * nI);
    auto k = dev::k_interp<T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k<<<n_items, 256, smem, st>>>(n_b, slot, parent, u, up, W);
    return cudaGetLastError();
}

}  // namespace lgf
