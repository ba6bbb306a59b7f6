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

#include <algorithm>
#include <cstring>

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
// Items (blocks or intervals) per CTA of the per-block transforms: small
// transforms share a CTA, so that its passes have lines for its threads (the
// level-0 transform of n_b = 8 has 9 x 8 y-lines: four blocks per CTA give
// 288).  A pass of one line per thread takes as many rounds as its lines
// need: with 256 threads the level-0 transform of n_b = 16 (17 x 16 y-lines,
// 17 x 32 z-lines) runs 2 + 3 rounds, with 272 threads 1 + 2.
template <typename T, int S, int N>
__host__ __device__ constexpr int fft_items_per_cta() {
    constexpr int y_lines = (S / 2 + 1) * N;
    int k = 1;
    while (2 * k * y_lines <= 320 && k < 16) k *= 2;
    return k;
}
// CTA size: one round of the y pass where that is at most 288 lines (two CTAs
// per SM for FP32: their registers are capped accordingly, 120 per thread at
// 272), else 256.
template <typename T, int S, int N>
__host__ __device__ constexpr int fft_threads() {
    constexpr int lines = fft_items_per_cta<T, S, N>() * (S / 2 + 1) * N;
    return lines <= 288 ? ((lines + 31) / 32 * 32 < 128 ? 128 : (lines + 31) / 32 * 32) : kFftThreads;
}
template <typename T, int S, int N>
__host__ __device__ constexpr int fft_min_blocks() {
    return sizeof(T) == 4 && fft_threads<T, S, N>() > kFftThreads ? 2 : 1;
}

// FP32 cubes whose rows are whole 16-byte vectors move between global memory
// and the x pass directly (each thread its own rows, 16-byte loads/stores),
// with no staged real cube in shared memory.
template <typename T, int N>
__host__ __device__ constexpr bool fft_direct_rows() {
    return sizeof(T) == 4 && N % 4 == 0;
}
// Shared-memory footprint of one item of the FFT kernels (bytes): the
// partially transformed cube with an odd row pitch, plus the staged real cube;
// and of a CTA (its items)
template <typename T, int S, int N>
__host__ __device__ constexpr size_t fft_item_smem() {
    return sizeof(cx<T>) * size_t(N) * ((S * ((S / 2 + 1) | 1)) | 1) +
           (fft_direct_rows<T, N>() ? 0 : sizeof(T) * size_t(N) * N * (N | 1));
}
template <typename T, int S, int N>
__host__ __device__ constexpr size_t fft_smem_bytes() {
    return fft_items_per_cta<T, S, N>() * fft_item_smem<T, S, N>();
}

// copy n reals (n % 4 == 0) with 16-byte vectors when both ends are aligned
template <typename T, typename F>
__device__ __forceinline__ void staged_copy(int n, const T* src, F&& put) {
    if (sizeof(T) == 4 && (n & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
        for (int i = threadIdx.x; i < n / 4; i += blockDim.x) {
            const float4 v = __ldg(s4 + i);
            put(4 * i, T(v.x));
            put(4 * i + 1, T(v.y));
            put(4 * i + 2, T(v.z));
            put(4 * i + 3, T(v.w));
        }
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) put(i, __ldg(src + i));
    }
}

// ---------------------------------------------------------------------------
// Padded R2C (Eq. alg_upfft): an NIN^3 real cube, zero-padded to S^3, to its
// half spectrum.  One CTA per item.  The input cube is first copied into
// shared memory with coalesced loads (rows of odd pitch RS).  The partially
// transformed cube stays in shared memory as B[(z*S + ky)*NXP + kx], z < NIN,
// NXP = NX rounded up to odd, so one-line-per-thread passes are free of bank
// conflicts; the last pass goes straight to global memory.
template <typename T, int S, int NIN>
__global__ void __launch_bounds__(fft_threads<T, S, NIN>(), fft_min_blocks<T, S, NIN>())
    k_r2c(const T* __restrict__ src, int64_t src_stride, const R2CItem* __restrict__ items,
          cx<T>* __restrict__ spec, int n_items) {
    constexpr int NX = S / 2 + 1, NXP = NX | 1, RS = NIN | 1, PP = (S * NXP) | 1;
    constexpr int64_t NWS = (int64_t(NX) * S * S + 31) / 32 * 32;
    constexpr int K = fft_items_per_cta<T, S, NIN>();
    constexpr size_t ITEM = fft_item_smem<T, S, NIN>();
    constexpr bool DIRECT = fft_direct_rows<T, NIN>();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ R2CItem its[K];
    const int first = blockIdx.x * K;
    const int nk = min(K, n_items - first);   // items of this CTA
    // one item: its indices in registers; several: in shared memory
    const R2CItem it0 = items[first];
    if constexpr (K > 1) {
        if (threadIdx.x < nk) its[threadIdx.x] = items[first + threadIdx.x];
        __syncthreads();
    }
    auto item = [&](int b) { return K == 1 ? it0 : its[b]; };
    // item b's partially transformed cube and staged input
    auto Bof = [&](int b) { return reinterpret_cast<cx<T>*>(smem_raw + b * ITEM); };
    auto Xof = [&](int b) { return reinterpret_cast<T*>(Bof(b) + NIN * PP); };
    auto in_of = [&](int b) { return src + int64_t(item(b).src) * src_stride; };
    // a kernel launched after this one with programmatic serialization (the
    // level-0 products) may start its prologue once every CTA got here; it
    // waits for this grid to finish before it reads the spectra
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if constexpr (!DIRECT) {
        for (int b = 0; b < nk; ++b) {
            T* X = Xof(b);
            staged_copy<T>(NIN * NIN * NIN, in_of(b), [&](int i, T v) { X[(i / NIN) * RS + i % NIN] = v; });
        }
        __syncthreads();
    }
    // x pass: lines l and l + NP (rows of the (y, z) plane) as one complex transform
    constexpr int NL = NIN * NIN, NP = (NL + 1) / 2;
    for (int p = threadIdx.x; p < (K == 1 ? NP : nk * NP); p += blockDim.x) {
        const int b = K == 1 ? 0 : p / NP, l0 = K == 1 ? p : p % NP, l1 = l0 + NP;
        const bool has1 = l1 < NL;
        cx<T>* B = Bof(b);
        cx<T> z[S];
        if constexpr (DIRECT) {
            // the two rows straight from global memory, 16-byte vectors when
            // the cube is 16-byte aligned (a caller's buffer may not be)
            const T* in = in_of(b);
            T a[NIN], c[NIN];
            const T* q0 = in + int64_t(l0) * NIN;
            const T* q1 = in + int64_t(has1 ? l1 : l0) * NIN;
            if ((reinterpret_cast<uintptr_t>(in) & 15) == 0) {
                const float4* g0 = reinterpret_cast<const float4*>(q0);
                const float4* g1 = reinterpret_cast<const float4*>(q1);
#pragma unroll
                for (int q = 0; q < NIN / 4; ++q) {
                    const float4 u = __ldg(g0 + q), v = __ldg(g1 + q);
                    a[4 * q] = u.x; a[4 * q + 1] = u.y; a[4 * q + 2] = u.z; a[4 * q + 3] = u.w;
                    c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int x = 0; x < NIN; ++x) {
                    a[x] = __ldg(q0 + x);
                    c[x] = __ldg(q1 + x);
                }
            }
#pragma unroll
            for (int x = 0; x < S; ++x) z[x] = x < NIN ? cx<T>{a[x], has1 ? c[x] : T(0)} : czero<T>();
        } else {
            const T* X = Xof(b);
            const T* r0 = X + l0 * RS;
            const T* r1 = X + (has1 ? l1 : l0) * RS;
#pragma unroll
            for (int x = 0; x < S; ++x)
                z[x] = x < NIN ? cx<T>{r0[x], has1 ? r1[x] : T(0)} : czero<T>();
        }
        fft<S, S, -1, NIN>(z);
        const int y0 = l0 % NIN, z0 = l0 / NIN, y1 = l1 % NIN, z1 = l1 / NIN;
        cx<T>* d0 = B + z0 * PP + y0 * NXP;
        cx<T>* d1 = B + z1 * PP + y1 * NXP;
#pragma unroll
        for (int k = 0; k < NX; ++k) {
            const cx<T> u = z[k], v = z[(S - k) % S];
            d0[k] = {T(0.5) * (u.x + v.x), T(0.5) * (u.y - v.y)};
            if (has1) d1[k] = {T(0.5) * (u.y + v.y), T(0.5) * (v.x - u.x)};
        }
    }
    __syncthreads();
    // y pass: lines (kx, z), in place within the column
    for (int q = threadIdx.x; q < (K == 1 ? NX * NIN : nk * NX * NIN); q += blockDim.x) {
        const int b = K == 1 ? 0 : q / (NX * NIN), l = K == 1 ? q : q % (NX * NIN);
        const int kx = l % NX, zz = l / NX;
        cx<T>* col = Bof(b) + zz * PP + kx;
        cx<T> v[S];
#pragma unroll
        for (int y = 0; y < S; ++y) v[y] = y < NIN ? col[y * NXP] : czero<T>();
        fft<S, S, -1, NIN>(v);
#pragma unroll
        for (int y = 0; y < S; ++y) col[y * NXP] = v[y];
    }
    __syncthreads();
    // z pass: lines (kx, ky), results to global (coalesced across the CTA)
    for (int q = threadIdx.x; q < (K == 1 ? NX * S : nk * NX * S); q += blockDim.x) {
        const int b = K == 1 ? 0 : q / (NX * S), l = K == 1 ? q : q % (NX * S);
        const int kx = l % NX, ky = l / NX;
        const cx<T>* col = Bof(b) + ky * NXP + kx;
        cx<T>* out = spec + int64_t(item(b).dst) * NWS;
        cx<T> v[S];
#pragma unroll
        for (int zz = 0; zz < S; ++zz) v[zz] = zz < NIN ? col[zz * PP] : czero<T>();
        fft<S, S, -1, NIN>(v);
#pragma unroll
        for (int kz = 0; kz < S; ++kz) out[int64_t(kz) * S * NX + l] = v[kz];
    }
}

// ---------------------------------------------------------------------------
// Truncated C2R (Eq. alg_dwfft): keep the first NOUT samples per axis.
//   dst[item.dst*dst_stride + (z*NOUT + y)*NOUT + x] = v (+ add[item.aux*add_stride
//   + (z*add_n + y)*add_n + x] when add != null and item.aux >= 0)
// The 1/S^3 of the inverse transform is folded into the kernel spectra.  The
// result cube is staged in shared memory (odd row pitch) and written with
// coalesced stores.
template <typename T, int S, int NOUT>
__global__ void __launch_bounds__(fft_threads<T, S, NOUT>(), fft_min_blocks<T, S, NOUT>())
    k_c2r(const cx<T>* __restrict__ spec, const C2RItem* __restrict__ items, T* __restrict__ dst,
          int64_t dst_stride, const T* __restrict__ add, int add_n, int64_t add_stride, int n_items) {
    constexpr int NX = S / 2 + 1, NXP = NX | 1, RS = NOUT | 1, PP = (S * NXP) | 1;
    constexpr int64_t NWS = (int64_t(NX) * S * S + 31) / 32 * 32;
    constexpr int K = fft_items_per_cta<T, S, NOUT>();
    constexpr size_t ITEM = fft_item_smem<T, S, NOUT>();
    constexpr bool DIRECT = fft_direct_rows<T, NOUT>();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ C2RItem its[K];
    const int first = blockIdx.x * K;
    const int nk = min(K, n_items - first);   // items of this CTA
    // one item: its indices in registers; several: in shared memory
    const C2RItem it0 = items[first];
    if constexpr (K > 1) {
        if (threadIdx.x < nk) its[threadIdx.x] = items[first + threadIdx.x];
        __syncthreads();
    }
    auto item = [&](int b) { return K == 1 ? it0 : its[b]; };
    auto Bof = [&](int b) { return reinterpret_cast<cx<T>*>(smem_raw + b * ITEM); };
    auto Oof = [&](int b) { return reinterpret_cast<T*>(Bof(b) + NOUT * PP); };
    auto out_of = [&](int b) { return dst + int64_t(item(b).dst) * dst_stride; };
    auto add_of = [&](int b) -> const T* {
        const int aux = item(b).aux;
        return (add != nullptr && aux >= 0) ? add + int64_t(aux) * add_stride : nullptr;
    };

    // z pass: lines (kx, ky); keep z < NOUT
    for (int q = threadIdx.x; q < (K == 1 ? NX * S : nk * NX * S); q += blockDim.x) {
        const int b = K == 1 ? 0 : q / (NX * S), l = K == 1 ? q : q % (NX * S);
        const int kx = l % NX, ky = l / NX;
        const cx<T>* in = spec + int64_t(item(b).src) * NWS;
        cx<T> v[S];
#pragma unroll
        for (int kz = 0; kz < S; ++kz) v[kz] = ldg_cx(in + int64_t(kz) * S * NX + l);
        fft<S, S, 1, S>(v);
        cx<T>* col = Bof(b) + ky * NXP + kx;
#pragma unroll
        for (int zz = 0; zz < NOUT; ++zz) col[zz * PP] = v[zz];
    }
    __syncthreads();
    // y pass: lines (kx, z < NOUT); keep y < NOUT
    for (int q = threadIdx.x; q < (K == 1 ? NX * NOUT : nk * NX * NOUT); q += blockDim.x) {
        const int b = K == 1 ? 0 : q / (NX * NOUT), l = K == 1 ? q : q % (NX * NOUT);
        const int kx = l % NX, zz = l / NX;
        cx<T>* col = Bof(b) + zz * PP + kx;
        cx<T> v[S];
#pragma unroll
        for (int y = 0; y < S; ++y) v[y] = col[y * NXP];
        fft<S, S, 1, S>(v);
#pragma unroll
        for (int y = 0; y < NOUT; ++y) col[y * NXP] = v[y];
    }
    __syncthreads();
    // x pass: two Hermitian half-lines (rows l and l + NP) per complex inverse
    constexpr int NL = NOUT * NOUT, NP = (NL + 1) / 2;
    for (int p = threadIdx.x; p < (K == 1 ? NP : nk * NP); p += blockDim.x) {
        const int b = K == 1 ? 0 : p / NP, l0 = K == 1 ? p : p % NP, l1 = l0 + NP;
        const bool has1 = l1 < NL;
        const cx<T>* B = Bof(b);
        const int y0 = l0 % NOUT, z0 = l0 / NOUT, y1 = l1 % NOUT, z1 = l1 / NOUT;
        const cx<T>* ra = B + z0 * PP + y0 * NXP;
        const cx<T>* rb = B + (has1 ? z1 : z0) * PP + (has1 ? y1 : y0) * NXP;
        cx<T> z[S];
#pragma unroll
        for (int k = 0; k < NX; ++k) {
            cx<T> A = ra[k], Bk = has1 ? rb[k] : czero<T>();
            if (k == 0 || 2 * k == S) {   // exactly real for a real signal
                A.y = T(0);
                Bk.y = T(0);
            }
            z[k] = {A.x - Bk.y, A.y + Bk.x};
            if (k > 0 && S - k >= NX) z[S - k] = {A.x + Bk.y, Bk.x - A.y};
        }
        fft<S, S, 1, S>(z);
        if constexpr (DIRECT) {
            // the two rows straight to global memory (plus the level-1 field),
            // 16-byte vectors when the output is 16-byte aligned
            T* out = out_of(b);
            const T* ad = add_of(b);
            const bool vec = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && !has1) break;
                const int l = h == 0 ? l0 : l1;
                T v[NOUT];
#pragma unroll
                for (int x = 0; x < NOUT; ++x) v[x] = h == 0 ? z[x].x : z[x].y;
                if (ad) {
                    const T* a = ad + ((l / NOUT) * add_n + l % NOUT) * add_n;
#pragma unroll
                    for (int x = 0; x < NOUT; ++x) v[x] += __ldg(a + x);
                }
                T* o = out + int64_t(l) * NOUT;
                if (vec) {
#pragma unroll
                    for (int q = 0; q < NOUT / 4; ++q)
                        reinterpret_cast<float4*>(o)[q] = make_float4(float(v[4 * q]), float(v[4 * q + 1]),
                                                                      float(v[4 * q + 2]), float(v[4 * q + 3]));
                } else {
#pragma unroll
                    for (int x = 0; x < NOUT; ++x) o[x] = v[x];
                }
            }
        } else {
            T* O = Oof(b);
#pragma unroll
            for (int x = 0; x < NOUT; ++x) {
                O[l0 * RS + x] = z[x].x;
                if (has1) O[l1 * RS + x] = z[x].y;
            }
        }
    }
    if constexpr (!DIRECT) {
        // the staged cubes out with coalesced stores, plus the level-1 field
        __syncthreads();
        constexpr int N3 = NOUT * NOUT * NOUT;
        for (int q = threadIdx.x; q < nk * N3; q += blockDim.x) {
            const int b = q / N3, i = q % N3;
            const int x = i % NOUT, yz = i / NOUT;
            const T* ad = add_of(b);
            T v = Oof(b)[yz * RS + x];
            if (ad) v += ad[((yz / NOUT) * add_n + yz % NOUT) * add_n + x];
            out_of(b)[i] = v;
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
                                                    int64_t NW, int64_t NWS) {
    const int64_t w = int64_t(blockIdx.y) * 32 + threadIdx.x;
    const int g = blockIdx.x * blockDim.y + threadIdx.y;
    if (g >= n_groups || w >= NW) return;
    cx<T> k[27];
#pragma unroll
    for (int d = 0; d < 27; ++d) k[d] = ldg_cx(kh + int64_t(d) * NWS + w);
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
                const cx<T> F = ldg_cx(fh + (int64_t(q) * 8 + cs) * NWS + w);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int dx = tx - (c & 1), dy = ty - ((c >> 1) & 1), dz = tz - (c >> 2);
                    if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) continue;
                    acc[c] = cmac(acc[c], F, k[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)]);
                }
            }
#pragma unroll
    for (int c = 0; c < 8; ++c) uh[(int64_t(g) * 8 + c) * NWS + w] = acc[c];
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
// mbarrier and bulk-copy helpers (inline PTX)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return done != 0;
}
// Waits for the phase with this parity to complete; false after about 2^32
// SM cycles (~2 s), far beyond any copy of this kernel.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(b, parity))
        if (clock64() - t0 > (1LL << 32)) return false;
    return true;
}
// bytes (multiple of 16) from global to this CTA's shared memory, both 16-byte
// aligned; completion counted on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 2D tensor-map copy of one box at element coordinates (x, y) into this
// CTA's shared memory (128-byte aligned), completion counted on bar
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// The 343-offset kernel tables store rows 171..342 only (kSymRows rows);
// row d < 171 is the complex conjugate of row 342 - d (offset -d).  A chunk's
// stored rows arrive as one tensor box into rows 171..342 of the chunk's
// shared-memory table, and the first 171 rows are filled by conjugation.
constexpr int kSymRows = 172, kSymFirst = 171;

template <typename T>
__device__ __forceinline__ cx<T> conjx(cx<T> v) { return {v.x, -v.y}; }

// coefficient of 7^3-table row d at frequency w, from the stored half table
template <typename T, int64_t NWS>
__device__ __forceinline__ cx<T> coef_sym(const cx<T>* __restrict__ kh, int d, int64_t w) {
    return d >= kSymFirst ? ldg_cx(kh + int64_t(d - kSymFirst) * NWS + w)
                          : conjx(ldg_cx(kh + int64_t(kSymFirst - d) * NWS + w));
}

// rows 0..170 of a [343][32] shared table from its rows 171..342
template <typename T>
__device__ __forceinline__ void mirror_rows(cx<T>* sk, int tid, int nthreads) {
    for (int i = tid; i < kSymFirst * 32; i += nthreads) {
        const int r = i >> 5, l = i & 31;
        sk[i] = conjx(sk[(2 * kSymFirst - r) * 32 + l]);
    }
}

// Tables reduced by the reflections of G (Sec. 3.2, last paragraph): G is even
// in each coordinate and symmetric in its arguments, so the kernel vector of
// offset d = (dx, dy, dz) is that of its representative r = (|dx|,
// min(|dy|, |dz|), max(|dy|, |dz|)) with the axes reflected (m_a -> s_a m_a,
// s_a the sign of d_a) and, when |dy| > |dz|, y and z exchanged.  The vector
// sits symmetrically about index 0 of the circular grid, so its spectrum is
// the representative's at the reflected and exchanged frequency, with no
// twiddle factor: khat_d(k) = khat_r(P S k), S = diag(s), P the y-z exchange.
// A reflected x frequency leaves the stored half (kx in [0, S/2]); there
// khat_r(-kx, ky', kz') = conj(khat_r(kx, -ky', -kz')) (real kernel vector).
// The 40 representatives (|dx| 0..3 times the 10 pairs a <= b of 0..3) are
// the rows of the reduced table, row 10 |dx| + b (b + 1) / 2 + a, instead of
// the 172 stored rows of the half table.
constexpr int kOctRows = 40;
__host__ __device__ constexpr int oct_row(int ax, int a, int b) { return 10 * ax + b * (b + 1) / 2 + a; }

// The coefficient rows 171..342 of frequencies w0 .. w0+31 gathered from the
// reduced table (the caller mirrors rows 0..170 by conjugation, as for the
// half table).  Each thread keeps one lane (one frequency) for every row it
// fills, so the frequency's reflected indices are computed once, and issues
// its gathers in batches of eight before storing them.
template <typename T, int S, int NT>
__device__ __forceinline__ void stage_coefficients_oct(cx<T>* __restrict__ sk, const cx<T>* __restrict__ kr,
                                                       int64_t w0, int tid) {
    constexpr int NX = S / 2 + 1;
    constexpr int64_t NW = int64_t(NX) * S * S, NWS = (NW + 31) / 32 * 32;
    constexpr int kRowsPerPass = NT / 32, kBatch = 8;
    static_assert(NT % 32 == 0, "whole warps");
    const int lane = tid & 31;
    const int64_t w = w0 + lane;
    const bool live = w < NW;
    const int wi = live ? int(w) : 0;
    const int kx = wi % NX, ky = (wi / NX) % S, kz = wi / (NX * S);
    const int nky = ky == 0 ? 0 : S - ky, nkz = kz == 0 ? 0 : S - kz;
    for (int base = kSymFirst + (tid >> 5); base < 343; base += kBatch * kRowsPerPass) {
        cx<T> v[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int row = base + j * kRowsPerPass;
            v[j] = czero<T>();
            if (row < 343 && live) {
                const int dx = row % 7 - 3, dy = (row / 7) % 7 - 3, dz = row / 49 - 3;
                const int ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
                const bool xneg = dx < 0, swap = ay > az;
                // signs applied to (ky, kz); a reflected x frequency folds back
                // with the y and z signs flipped and the value conjugated
                const bool fy = (dy < 0) != xneg, fz = (dz < 0) != xneg;
                const int ky1 = fy ? nky : ky, kz1 = fz ? nkz : kz;
                const int kyy = swap ? kz1 : ky1, kzz = swap ? ky1 : kz1;
                const int r = oct_row(xneg ? -dx : dx, swap ? az : ay, swap ? ay : az);
                v[j] = ldg_cx(kr + int64_t(r) * NWS + (int64_t(kzz) * S + kyy) * NX + kx);
                if (xneg) v[j] = conjx(v[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int row = base + j * kRowsPerPass;
            if (row < 343) sk[row * 32 + lane] = v[j];
        }
    }
}

// Packed form of the 8 x 8 sibling products (fma.rn.f32x2: two FP32 FMAs per
// instruction).  With F = Fx + i Fy and K = Kx + i Ky, A accumulates
// (Fx Kx, Fx Ky) and B accumulates (Fy Kx, Fy Ky), both against K as stored;
// the complex sum is (A.x - B.y) + i (A.y + B.x).  Half the FMA instructions
// of persist_block for the same coefficient loads.
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void ffma2(uint64_t& d, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
__device__ __forceinline__ cx<float> unpack_sum(uint64_t A, uint64_t B) {
    float ax, ay, bx, by;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(ax), "=f"(ay) : "l"(A));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(bx), "=f"(by) : "l"(B));
    return {ax - by, ay + bx};
}
// The 27 coefficients of one source group come as three x-planes of 9 (dy,
// dz) values: plane dx holds rows centre + dx + 7 dy + 49 dz.  A source group
// that is the +x neighbour (centre row + 2) of the previous pair's shares its
// -x plane with that pair's +x plane.  The pair loop keeps three plane
// register sets whose roles rotate between its two unrolled halves, so the
// shared plane is reused in place: adjacency only skips its 9 loads.
__device__ __forceinline__ void persist_plane(uint64_t (&P)[9], const cx<float>* kb) {
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
            P[(dy + 1) + 3 * (dz + 1)] = *reinterpret_cast<const uint64_t*>(kb + (7 * dy + 49 * dz) * 32);
}
// the 8 x 8 sibling products of one source group from its -x, centre and +x
// coefficient planes L, M, R
__device__ __forceinline__ void persist_block_packed(uint64_t (&A)[8], uint64_t (&B)[8], const cx<float> (&F)[8],
                                                     const uint64_t (&L)[9], const uint64_t (&M)[9],
                                                     const uint64_t (&R)[9]) {
#pragma unroll
    for (int cs = 0; cs < 8; ++cs) {
        const uint64_t fx = pk2(F[cs].x, F[cs].x), fy = pk2(F[cs].y, F[cs].y);
#pragma unroll
        for (int ct = 0; ct < 8; ++ct) {
            const int dx = (cs & 1) - (ct & 1), dy = ((cs >> 1) & 1) - ((ct >> 1) & 1), dz = (cs >> 2) - (ct >> 2);
            const int i = (dy + 1) + 3 * (dz + 1);
            const uint64_t k = dx < 0 ? L[i] : dx == 0 ? M[i] : R[i];
            ffma2(A[ct], fx, k);
            ffma2(B[ct], fy, k);
        }
    }
}

constexpr int kMacWarps = 12;
constexpr int kMacPackedWarps = 8;   // packed form: 128 registers for two CTAs per SM

// One warp's walk over the (group, neighbour) pairs it owns: groups
// g0 + warp, g0 + warp + kMacWarps, ... below g1, and for each group the
// present neighbour groups e != 13 in increasing order.
struct MacWalk {
    int g, e;            // current pair (g: position in the work order; e < 0: no neighbours)
    int gid;             // group id at position g
    unsigned mask;       // neighbours of gid not yet visited
    int self;            // whether the group's own block (e = 13) is a source
};

// present neighbour groups; the group itself (e = 13) only when include_self
__device__ __forceinline__ unsigned nbr_mask(const int* __restrict__ gnbr, int g, int include_self = 0) {
    const int* nb = gnbr + int64_t(g) * 27;
    unsigned m = 0;
#pragma unroll
    for (int e = 0; e < 27; ++e)
        if ((e != 13 || include_self) && __ldg(nb + e) >= 0) m |= 1u << e;
    return m;
}

// advance to the next pair; returns false past the warp's last group
template <int WARPS = kMacWarps>
__device__ __forceinline__ bool mac_next(MacWalk& it, const int* __restrict__ gnbr, const int* __restrict__ order,
                                         int g1) {
    if (it.mask) {
        it.e = __ffs(it.mask) - 1;
        it.mask &= it.mask - 1;
        return true;
    }
    it.g += WARPS;
    if (it.g >= g1) return false;
    it.gid = __ldg(order + it.g);
    it.mask = nbr_mask(gnbr, it.gid, it.self);
    if (it.mask) {
        it.e = __ffs(it.mask) - 1;
        it.mask &= it.mask - 1;
    } else {
        it.e = -1;
    }
    return true;
}

template <typename T, int S>
__device__ __forceinline__ void mac_load(cx<T> (&F)[8], const cx<T>* __restrict__ fh,
                                         const int* __restrict__ gnbr, const MacWalk& it, int64_t wc) {
    constexpr int64_t NWS = (int64_t(S / 2 + 1) * S * S + 31) / 32 * 32;
    if (it.e < 0) return;
    const cx<T>* src = fh + int64_t(__ldg(gnbr + int64_t(it.gid) * 27 + it.e)) * (8 * NWS) + wc;
#pragma unroll
    for (int c = 0; c < 8; ++c) F[c] = ldg_cx(src + c * NWS);
}

template <typename T>
__device__ __forceinline__ void mac_block(cx<T> (&acc)[8], const cx<T> (&F)[8], const cx<T>* __restrict__ sk,
                                          int e) {
    // centre offset d = 2e of this neighbour in the 7^3 coefficient rows
    const int ex = e % 3, ey = (e / 3) % 3, ez = e / 9;      // 0..2
    const cx<T>* kb = sk + ((2 * ex + 1) + 7 * (2 * ey + 1) + 49 * (2 * ez + 1)) * 32 + threadIdx.x;
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
            const int dx = (cs & 1) - (ct & 1), dy = ((cs >> 1) & 1) - ((ct >> 1) & 1), dz = (cs >> 2) - (ct >> 2);
            acc[ct] = cmac(acc[ct], F[cs], kk[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)]);
        }
}

// Packed form of mac_block (FP32): the three coefficient planes of the
// neighbour's centre and the packed 8 x 8 products (persist_block_packed).
__device__ __forceinline__ void mac_block_packed(uint64_t (&A)[8], uint64_t (&B)[8], const cx<float> (&F)[8],
                                                 const cx<float>* __restrict__ sk, int e) {
    const int ex = e % 3, ey = (e / 3) % 3, ez = e / 9;
    const cx<float>* kb = sk + ((2 * ex + 1) + 7 * (2 * ey + 1) + 49 * (2 * ez + 1)) * 32 + threadIdx.x;
    uint64_t L[9], M[9], R[9];
    persist_plane(L, kb - 32);
    persist_plane(M, kb);
    persist_plane(R, kb + 32);
    persist_block_packed(A, B, F, L, M, R);
}

// The 343 coefficient rows of the frequencies w0 .. w0+31 into shared memory
// ([343][32], zero past NW) from the stored half table: eight independent
// loads per thread in flight before their stores, so a CTA keeps enough
// requests outstanding to stream.
template <typename T, int64_t NW, int64_t NWS, int NT>
__device__ __forceinline__ void stage_coefficients(cx<T>* __restrict__ sk, const cx<T>* __restrict__ kh, int64_t w0,
                                                   int tid) {
    constexpr int kTotal = 343 * 32, kBatch = 8;
    for (int base = 0; base < kTotal; base += kBatch * NT) {
        cx<T> v[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int i = base + j * NT + tid;
            const int64_t w = w0 + (i & 31);
            v[j] = (i < kTotal && w < NW) ? coef_sym<T, NWS>(kh, i >> 5, w) : czero<T>();
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int i = base + j * NT + tid;
            if (i < kTotal) sk[i] = v[j];
        }
    }
}

// Groups are visited in the plan's work order (sorted by neighbour count, so
// the warps of one CTA carry similar work).  With include_self the group's own
// sibling block e = 13 is a source too: that is the merged level-0 / level-1
// form, where the 343 coefficient rows hold the near offsets as well.
template <typename T, int S, int WARPS = kMacWarps, bool PACKED = false>
__global__ void __launch_bounds__(32 * WARPS, sizeof(T) == 4 ? 2 : 1) k_mac_interval(const cx<T>* __restrict__ fh,
                                                                   const cx<T>* __restrict__ kh,
                                                                   cx<T>* __restrict__ uh,
                                                                   const int* __restrict__ gnbr,
                                                                   const int* __restrict__ order, int n_groups,
                                                                   int groups_per_cta, int include_self,
                                                                   const __grid_constant__ CUtensorMap tmap,
                                                                   int use_tma, int* __restrict__ err, int oct) {
    constexpr int64_t NW = int64_t(S / 2 + 1) * S * S;
    constexpr int64_t NWS = (NW + 31) / 32 * 32;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    cx<T>* sk = reinterpret_cast<cx<T>*>(smem_raw);   // [343][32]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + sizeof(cx<T>) * 343 * 32);
    const int64_t w0 = int64_t(blockIdx.y) * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (oct) {
        // the reflection-reduced table: the stored half's rows gathered by
        // their frequency maps, the other half by conjugation
        stage_coefficients_oct<T, S, 32 * WARPS>(sk, kh, w0, tid);
        __syncthreads();
        mirror_rows(sk, tid, 32 * WARPS);
        __syncthreads();
    } else if (use_tma) {
        // the chunk's stored rows as one tensor box (x in reals: 2 per complex)
        if (tid == 0) {
            mbar_init(bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            mbar_expect_tx(bar, unsigned(sizeof(cx<T>) * kSymRows * 32));
            tma_2d(sk + kSymFirst * 32, &tmap, int(2 * w0), 0, bar);
        }
        __syncthreads();
        if (!mbar_wait(bar, 0)) {
            if (tid == 0) atomicExch(err, 1);
            return;
        }
        mirror_rows(sk, tid, 32 * WARPS);
        __syncthreads();
    } else {
        stage_coefficients<T, NW, NWS, 32 * WARPS>(sk, kh, w0, tid);
        __syncthreads();
    }
    const int g0 = blockIdx.x * groups_per_cta;
    const int g1 = min(n_groups, g0 + groups_per_cta);
    const int64_t w = w0 + threadIdx.x;
    const int64_t wc = w < NW ? w : NW - 1;
    MacWalk cur{g0 + int(threadIdx.y) - WARPS, -1, 0, 0u, include_self};
    if (!mac_next<WARPS>(cur, gnbr, order, g1)) return;
    cx<T> Fa[8], Fb[8], acc[8];
    [[maybe_unused]] uint64_t A[8], B[8];   // packed form (FP32)
    auto zero = [&] {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            acc[c] = czero<T>();
            if constexpr (PACKED) A[c] = B[c] = 0ull;
        }
    };
    auto block = [&](const cx<T> (&F)[8], int e) {
        if constexpr (PACKED) mac_block_packed(A, B, F, sk, e);
        else mac_block(acc, F, sk, e);
    };
    // the group's sums out, accumulators cleared
    auto flush = [&](int gid) {
        if constexpr (PACKED) {
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = unpack_sum(A[c], B[c]);
        }
        if (w < NW) {
#pragma unroll
            for (int c = 0; c < 8; ++c) uh[(int64_t(gid) * 8 + c) * NWS + w] = acc[c];
        }
        zero();
    };
    zero();
    mac_load<T, S>(Fa, fh, gnbr, cur, wc);
    // two pairs per trip so the prefetch buffers alternate without copies
    while (true) {
        MacWalk nxt = cur;
        bool more = mac_next<WARPS>(nxt, gnbr, order, g1);
        if (more) mac_load<T, S>(Fb, fh, gnbr, nxt, wc);
        if (cur.e >= 0) block(Fa, cur.e);
        if (!more || nxt.g != cur.g) flush(cur.gid);
        if (!more) break;
        cur = nxt;
        nxt = cur;
        more = mac_next<WARPS>(nxt, gnbr, order, g1);
        if (more) mac_load<T, S>(Fa, fh, gnbr, nxt, wc);
        if (cur.e >= 0) block(Fb, cur.e);
        if (!more || nxt.g != cur.g) flush(cur.gid);
        if (!more) break;
        cur = nxt;
    }
}

// ---------------------------------------------------------------------------
// Interaction-list products, two groups per warp.  The bound of the
// one-group form is the shared-memory/L1 data path: 27 coefficient loads per
// 64 products.  Here a warp walks two Morton-adjacent groups A, B together,
// over the union of their neighbour offsets e; the 27 coefficients of e are
// loaded once and applied to A's and B's source blocks (each only if that
// group has neighbour e, a warp-uniform test), which halves coefficient
// traffic per product.  One CTA of kMacPWarps warps per SM (FP32 registers).
constexpr int kMacPWarps = 16;

template <typename T, int S>
__device__ __forceinline__ void macp_load(cx<T> (&F)[8], const cx<T>* __restrict__ fh, int q, int64_t wc) {
    constexpr int64_t NWS = (int64_t(S / 2 + 1) * S * S + 31) / 32 * 32;
    const cx<T>* src = fh + int64_t(q) * (8 * NWS) + wc;
#pragma unroll
    for (int c = 0; c < 8; ++c) F[c] = ldg_cx(src + c * NWS);
}

// Products of one neighbour offset e for groups A and B (each if present),
// the 27 coefficients read in three slices of fixed dz = cs_z - ct_z so that
// only 9 are live at a time.
template <typename T>
__device__ __forceinline__ void macp_pair_block(cx<T> (&accA)[8], const cx<T> (&FA)[8], bool hasA,
                                                cx<T> (&accB)[8], const cx<T> (&FB)[8], bool hasB,
                                                const cx<T>* __restrict__ sk, int e) {
    const int ex = e % 3, ey = (e / 3) % 3, ez = e / 9;
    const cx<T>* kb = sk + ((2 * ex + 1) + 7 * (2 * ey + 1) + 49 * (2 * ez + 1)) * 32 + threadIdx.x;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        cx<T> kk[9];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) kk[(dx + 1) + 3 * (dy + 1)] = kb[(dx + 7 * dy + 49 * dz) * 32];
#pragma unroll
        for (int ct = 0; ct < 8; ++ct)
#pragma unroll
            for (int cs = 0; cs < 8; ++cs) {
                if ((cs >> 2) - (ct >> 2) != dz) continue;
                const int dx = (cs & 1) - (ct & 1), dy = ((cs >> 1) & 1) - ((ct >> 1) & 1);
                const cx<T> kv = kk[(dx + 1) + 3 * (dy + 1)];
                if (hasA) accA[ct] = cmac(accA[ct], FA[cs], kv);
                if (hasB) accB[ct] = cmac(accB[ct], FB[cs], kv);
            }
    }
}

template <typename T, int S>
__global__ void __launch_bounds__(32 * kMacPWarps, 1) k_mac_interval_pair(const cx<T>* __restrict__ fh,
                                                                         const cx<T>* __restrict__ kh,
                                                                         cx<T>* __restrict__ uh,
                                                                         const int* __restrict__ gnbr,
                                                                         const int* __restrict__ order,
                                                                         int n_groups, int groups_per_cta,
                                                                         int include_self) {
    constexpr int64_t NW = int64_t(S / 2 + 1) * S * S;
    constexpr int64_t NWS = (NW + 31) / 32 * 32;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    cx<T>* sk = reinterpret_cast<cx<T>*>(smem_raw);   // [343][32]
    const int64_t w0 = int64_t(blockIdx.y) * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    stage_coefficients<T, NW, NWS, 32 * kMacPWarps>(sk, kh, w0, tid);
    __syncthreads();
    const int g0 = blockIdx.x * groups_per_cta;
    const int g1 = min(n_groups, g0 + groups_per_cta);
    const int64_t w = w0 + threadIdx.x;
    const int64_t wc = w < NW ? w : NW - 1;
    for (int pa = g0 + 2 * int(threadIdx.y); pa < g1; pa += 2 * kMacPWarps) {
        const int ga = __ldg(order + pa);
        const int gb = pa + 1 < g1 ? __ldg(order + pa + 1) : -1;
        const unsigned ma = nbr_mask(gnbr, ga, include_self);
        const unsigned mb = gb >= 0 ? nbr_mask(gnbr, gb, include_self) : 0u;
        unsigned mask = ma | mb;
        cx<T> accA[8], accB[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            accA[c] = czero<T>();
            accB[c] = czero<T>();
        }
        if (mask) {
            int e = __ffs(mask) - 1;
            mask &= mask - 1;
            cx<T> FA[8], FB[8];
            if ((ma >> e) & 1) macp_load<T, S>(FA, fh, __ldg(gnbr + int64_t(ga) * 27 + e), wc);
            if ((mb >> e) & 1) macp_load<T, S>(FB, fh, __ldg(gnbr + int64_t(gb) * 27 + e), wc);
            while (true) {
                const int en = mask ? __ffs(mask) - 1 : -1;
                mask &= mask - 1;
                cx<T> NA[8], NB[8];
                if (en >= 0 && ((ma >> en) & 1)) macp_load<T, S>(NA, fh, __ldg(gnbr + int64_t(ga) * 27 + en), wc);
                if (en >= 0 && ((mb >> en) & 1)) macp_load<T, S>(NB, fh, __ldg(gnbr + int64_t(gb) * 27 + en), wc);
                macp_pair_block(accA, FA, ((ma >> e) & 1) != 0, accB, FB, ((mb >> e) & 1) != 0, sk, e);
                if (en < 0) break;
                e = en;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    FA[c] = NA[c];
                    FB[c] = NB[c];
                }
            }
        }
        if (w < NW) {
#pragma unroll
            for (int c = 0; c < 8; ++c) uh[(int64_t(ga) * 8 + c) * NWS + w] = accA[c];
            if (gb >= 0) {
#pragma unroll
                for (int c = 0; c < 8; ++c) uh[(int64_t(gb) * 8 + c) * NWS + w] = accB[c];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent interaction kernel (FP32).  The same sums as k_mac_interval, with
// one CTA per SM working through a contiguous range of units (frequency chunk
// of 32, group position) fixed at plan time so every CTA carries the same
// number of (group, source) pairs.  The 343 coefficient rows of a chunk
// (87.8 KB) arrive in shared memory by bulk copies (cp.async.bulk, completion
// on an mbarrier) into one of two buffers, so the next chunk loads while the
// current one is used; warps take groups of the current chunk from a shared
// counter, and the last warp to finish a chunk refills its buffer with the
// chunk after next.  Each group's sources come from a flat list (source group,
// centre coefficient row), so the inner loop has no neighbour-mask logic.
constexpr int kPersistWarps = 24;
constexpr int kPersistWarpsPacked = 16;   // the packed form holds more registers

__device__ __forceinline__ PairSrc ldg_pair(const PairSrc* p) {
    const int2 v = __ldg(reinterpret_cast<const int2*>(p));
    return {v.x, v.y};
}

template <int S>
__device__ __forceinline__ void persist_load(cx<float> (&F)[8], const cx<float>* __restrict__ fh, int src,
                                             int64_t wc) {
    constexpr int64_t NWS = (int64_t(S / 2 + 1) * S * S + 31) / 32 * 32;
    const cx<float>* p = fh + int64_t(src) * (8 * NWS) + wc;
#pragma unroll
    for (int c = 0; c < 8; ++c) F[c] = ldg_cx(p + c * NWS);
}

// the 8 x 8 sibling products of one source group; kb: centre row of this lane
__device__ __forceinline__ void persist_block(cx<float> (&acc)[8], const cx<float> (&F)[8],
                                              const cx<float>* kb) {
    cx<float> kk[27];
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
            const int dx = (cs & 1) - (ct & 1), dy = ((cs >> 1) & 1) - ((ct >> 1) & 1), dz = (cs >> 2) - (ct >> 2);
            acc[ct] = cmac(acc[ct], F[cs], kk[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)]);
        }
}

// Store of a product spectrum value with an L2 evict-last policy: the level-0
// inverse FFT reads these spectra right after the launch, and the launch's own
// traffic (source spectra, coefficient chunks) would otherwise push them out.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_keep(cx<float>* p, cx<float> v, uint64_t policy) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(policy)
                 : "memory");
}

constexpr unsigned kPersistBuf = 343u * 32u * sizeof(cx<float>);   // bytes per coefficient buffer
constexpr unsigned kPersistFill = unsigned(kSymRows) * 32u * sizeof(cx<float>);   // bytes copied per chunk
constexpr size_t kPersistSmem = 2 * size_t(kPersistBuf) + 64;

template <int S, int WARPS, bool PACKED>
__global__ void __launch_bounds__(32 * WARPS, 1)
    k_mac_persist(const cx<float>* __restrict__ fh, const cx<float>* __restrict__ kh, cx<float>* __restrict__ uh,
                  const PairSrc* __restrict__ pairs, const int* __restrict__ start, const int* __restrict__ order,
                  const long long* __restrict__ cta_units, int n_groups, int* __restrict__ err,
                  const __grid_constant__ CUtensorMap tmap, int use_tma) {
    constexpr int64_t NW = int64_t(S / 2 + 1) * S * S;
    constexpr int64_t NWS = (NW + 31) / 32 * 32;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    cx<float>* buf = reinterpret_cast<cx<float>*>(smem_raw);                 // [2][343][32]
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + 2 * kPersistBuf);   // [2] copy landed
    uint64_t* ready = full + 2;                                                // [2] rows mirrored
    int* ctr = reinterpret_cast<int*>(ready + 2);                            // [2] next position
    int* done = ctr + 2;                                                     // [2] warps finished
    // this CTA's work: whole chunks [m0, m1), then the units [r0, r1) of the
    // chunks left over (unit = chunk * n_groups + position); visit j is the
    // j-th chunk of that sequence with its positions [pb, pe)
    const long long* cu = cta_units + 4 * int64_t(blockIdx.x);
    const long long m0 = cu[0], m1 = cu[1], r0 = cu[2], r1 = cu[3];
    const int nm = int(m1 - m0);
    const long long rc0 = r1 > r0 ? r0 / n_groups : 0, rc1 = r1 > r0 ? (r1 - 1) / n_groups : -1;
    const int V = nm + int(rc1 - rc0 + 1);
    if (V <= 0) return;
    auto chunk_of = [&](int j) -> long long { return j < nm ? m0 + j : rc0 + (j - nm); };
    const int warp = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    const uint64_t keep = l2_evict_last_policy();
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&ready[0], 1);
        mbar_init(&ready[1], 1);
        ctr[0] = ctr[1] = 0;
        done[0] = done[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // one warp loads visit j's chunk: the stored rows by one tensor box (or
    // 172 row copies), then, once they landed, the mirrored rows by
    // conjugation; ready[b] releases the chunk to every warp
    auto issue = [&](int j) {
        const int b = j & 1;
        const long long c = chunk_of(j);
        cx<float>* dst = buf + b * (343 * 32) + kSymFirst * 32;
        if (use_tma) {
            if (lane == 0) {
                mbar_expect_tx(&full[b], kPersistFill);
                tma_2d(dst, &tmap, int(c * 64), 0, &full[b]);
            }
            return;
        }
        if (lane == 0) mbar_expect_tx(&full[b], kPersistFill);
        __syncwarp();
        const cx<float>* src = kh + c * 32;
        for (int r = lane; r < kSymRows; r += 32) bulk_g2s(dst + r * 32, src + int64_t(r) * NWS, 256u, &full[b]);
    };
    auto finish = [&](int j) {
        const int b = j & 1;
        if (mbar_wait(&full[b], unsigned((j >> 1) & 1))) {
            cx<float>* t = buf + b * (343 * 32);
            for (int r = 0; r < kSymFirst; ++r) t[r * 32 + lane] = conjx(t[(2 * kSymFirst - r) * 32 + lane]);
        } else if (lane == 0) {
            atomicExch(err, 1);
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ready[b])) : "memory");
    };
    if (warp == 0) {
        issue(0);
        if (V > 1) issue(1);
        finish(0);
        if (V > 1) finish(1);
    }
    // launched early behind the forward FFT (programmatic serialization): the
    // coefficient staging above needs only the kernel tables; the source
    // spectra are read after the FFT's grid has completed (a no-op otherwise)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int j = 0; j < V; ++j) {
        const int b = j & 1;
        if (!mbar_wait(&ready[b], unsigned((j >> 1) & 1))) {
            if (lane == 0) atomicExch(err, 1);
            return;
        }
        const long long c = chunk_of(j);
        const cx<float>* sk = buf + b * (343 * 32) + lane;
        const int pb = j >= nm && c == rc0 ? int(r0 % n_groups) : 0;
        const int pe = j >= nm && c == rc1 ? int((r1 - 1) % n_groups) + 1 : n_groups;
        const int64_t w = c * 32 + lane;
        const int64_t wc = w < NW ? w : NW - 1;
        while (true) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&ctr[b], 1);
            const int pos = pb + __shfl_sync(0xffffffffu, k, 0);
            if (pos >= pe) break;
            const int p0 = __ldg(start + pos), p1 = __ldg(start + pos + 1);
            cx<float> acc[8];
            [[maybe_unused]] uint64_t A[8], B[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[i] = czero<float>();
                if constexpr (PACKED) A[i] = B[i] = 0ull;
            }
            // packed form: plane sets X, Y, Z; the first pair of an iteration
            // takes (L, M, R) = (X, Y, Z), the second (Z, Y, X), so a +x
            // neighbour finds its -x plane where the previous pair left its +x
            [[maybe_unused]] uint64_t X[9], Y[9], Z[9];
            int prev = -100;   // centre row of the previous pair of this group
            if (p1 > p0) {
                cx<float> Fa[8], Fb[8];
                PairSrc pa = ldg_pair(pairs + p0), pq{0, 0};
                persist_load<S>(Fa, fh, pa.src, wc);
                for (int p = p0;; p += 2) {
                    const bool hb = p + 1 < p1;
                    if (hb) {
                        pq = ldg_pair(pairs + p + 1);
                        persist_load<S>(Fb, fh, pq.src, wc);
                    }
                    if constexpr (PACKED) {
                        const cx<float>* kb = sk + pa.centre * 32;
                        if (pa.centre != prev + 2) persist_plane(X, kb - 32);
                        persist_plane(Y, kb);
                        persist_plane(Z, kb + 32);
                        persist_block_packed(A, B, Fa, X, Y, Z);
                        prev = pa.centre;
                    } else {
                        persist_block(acc, Fa, sk + pa.centre * 32);
                    }
                    if (!hb) break;
                    const bool ha = p + 2 < p1;
                    if (ha) {
                        pa = ldg_pair(pairs + p + 2);
                        persist_load<S>(Fa, fh, pa.src, wc);
                    }
                    if constexpr (PACKED) {
                        const cx<float>* kb = sk + pq.centre * 32;
                        if (pq.centre != prev + 2) persist_plane(Z, kb - 32);
                        persist_plane(Y, kb);
                        persist_plane(X, kb + 32);
                        persist_block_packed(A, B, Fb, Z, Y, X);
                        prev = pq.centre;
                    } else {
                        persist_block(acc, Fb, sk + pq.centre * 32);
                    }
                    if (!ha) break;
                }
            }
            if constexpr (PACKED) {
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = unpack_sum(A[i], B[i]);
            }
            if (w < NW) {
                cx<float>* out = uh + int64_t(__ldg(order + pos)) * (8 * NWS) + w;
#pragma unroll
                for (int i = 0; i < 8; ++i) st_keep(out + i * NWS, acc[i], keep);
            }
        }
        // this warp is done with visit j; the last one out refills the buffer
        // with visit j + 2 (every read of the buffer has completed by then)
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&done[b], 1) == WARPS - 1;
        }
        if (__shfl_sync(0xffffffffu, last, 0)) {
            if (lane == 0) {
                ctr[b] = 0;
                done[b] = 0;
            }
            if (j + 2 < V) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(j + 2);
                finish(j + 2);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Level-0 transforms as persistent kernels (FP32; NIN = NOUT = S/2, S % 4 ==
// 0).  One CTA per SM takes blocks from a counter.  Every pass splits its
// line transforms into output classes (decimation in frequency), so all warps
// of the CTA have work in every pass: a class-r task computes X[R m + r] of a
// length-S line from the R input blocks of length S/R folded with W_R^{r q},
// twisted by W_S^{r n}, and one length-S/R transform.
//  R2C (Eq. alg_upfft): the NIN^2 input rows arrive as one tensor box while
//  the previous block runs, 16-byte chunks swizzled per row (the tensor map's
//  swizzle of NIN * 4 bytes), so the x pass reads whole rows without bank
//  conflicts; x pass (two rows as one complex line, classes
//  kx even/odd) into a row buffer; y pass (ky even/odd) into the z-input
//  region; z pass even kz into the other region, stored by bulk copies while
//  the odd kz are computed in place and stored in turn.  The two regions swap
//  roles every block, so each store drains behind the next block's passes;
//  the per-SM write path, not the arithmetic, bounds this kernel.
//  C2R (Eq. alg_dwfft): the spectrum arrives by two bulk copies (planes NOUT
//  and up after the z pass is done with them, the rest after the y pass);
//  z pass in place, y pass (y even/odd) into a row buffer, x pass (x mod 4)
//  into the output cube, which is written with the level-1 field added.
// ctr[0] hands out blocks, ctr[1] counts CTAs that are done: the last one
// resets both, so the next launch starts from zero.  A wait that runs out sets
// err and ends the CTA.
// y-pass lines per class rounded up to whole warps, so each warp has one class
template <int S>
__host__ __device__ constexpr int cube_ycls() {
    return ((S / 2 + 1) * (S / 2) + 31) / 32 * 32;
}
template <int S>
__host__ __device__ constexpr int cube_threads() {
    return 2 * cube_ycls<S>() > (S / 2 + 1) * S ? 2 * cube_ycls<S>() : ((S / 2 + 1) * S + 31) / 32 * 32;
}
template <int S, int NIN>
__host__ __device__ constexpr size_t r2c_cube_smem() {
    return size_t(S) * S * (S / 2 + 1) * sizeof(cx<float>)                    // two regions of S/2 planes
           + size_t(NIN) * NIN * ((S / 2 + 1) | 1) * sizeof(cx<float>)     // x-pass rows
           + size_t(NIN) * NIN * NIN * sizeof(float) + 1024 + 64;           // swizzled input (1024-aligned)
}
template <int S, int NOUT>
__host__ __device__ constexpr size_t c2r_cube_smem() {
    return size_t(S) * S * (S / 2 + 1) * sizeof(cx<float>)                    // the spectrum
           + size_t(NOUT) * NOUT * ((S / 2 + 1) | 1) * sizeof(cx<float>)   // y-pass rows
           + size_t(NOUT) * NOUT * (NOUT | 1) * sizeof(float) + 64;         // output cube
}

// Class r of a length-S DFT with sign SIGN: out[m] = X[R m + r], m < S/R, of
// the N inputs x (zero from N on; N a multiple of S/R).
template <int S, int R, int r, int SIGN, int N>
__device__ __forceinline__ void dft_class(const cx<float> (&x)[N], cx<float> (&out)[S / R]) {
    constexpr int L = S / R;
    static_assert(S % R == 0 && N % L == 0 && N <= S, "input blocks of length S/R");
#pragma unroll
    for (int n = 0; n < L; ++n) {
        cx<float> v = x[n];
#pragma unroll
        for (int q = 1; q < N / L; ++q) v = v + twmul<S, SIGN>(x[n + q * L], r * q * L);
        out[n] = twmul<S, SIGN>(v, r * n);
    }
    fft<S, L, SIGN, L>(out);
}

// shared -> global bulk store (both 16-byte aligned, bytes % 16 == 0) in the
// issuing thread's current bulk group
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most N of this thread's bulk groups still reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// every bulk group of this thread complete (writes performed)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// thread 0, after its last claim
__device__ __forceinline__ void cube_done(int* ctr) {
    __threadfence();
    if (atomicAdd(ctr + 1, 1) == int(gridDim.x) - 1) {
        atomicExch(ctr, 0);
        atomicExch(ctr + 1, 0);
    }
}

// in_map: the input as rows of NIN reals (row = block * NIN^2 + z * NIN + y),
// box NIN x NIN^2, swizzle of NIN * 4 bytes (64B for NIN = 16, 32B for 8)
template <int S, int NIN>
__global__ void __launch_bounds__(cube_threads<S>(), 1)
    k_r2c_cube(const __grid_constant__ CUtensorMap in_map, const R2CItem* __restrict__ items, int n_items,
               cx<float>* __restrict__ spec, int* __restrict__ ctr, int* __restrict__ err) {
    constexpr int NX = S / 2 + 1, PP = S * NX, H = S / 2, NL = NIN * NIN, NP = NL / 2;
    constexpr int RP = NX | 1, YC = cube_ycls<S>();   // x-pass row pitch (complex): odd
    constexpr int64_t NWS = (int64_t(PP) * S + 31) / 32 * 32;
    constexpr unsigned PLANE = PP * unsigned(sizeof(cx<float>)), ROWB = NIN * 4u, SWZ = ROWB / 16 - 1;
    static_assert(NIN == H && S % 4 == 0 && (NIN == 16 || NIN == 8) && PP % 2 == 0,
                  "64B or 32B swizzled rows; bulk copies move 16-byte multiples");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    cx<float>* P = reinterpret_cast<cx<float>*>(smem_raw);   // [2][H planes]
    cx<float>* XB = P + S * PP;                               // [NL rows][RP]
    const uintptr_t xa = (reinterpret_cast<uintptr_t>(XB + NL * RP) + 1023) & ~uintptr_t(1023);
    const unsigned char* X = reinterpret_cast<const unsigned char*>(xa);   // [NL rows][ROWB], swizzled
    uint64_t* full = reinterpret_cast<uint64_t*>(xa + NL * ROWB);
    int* sh = reinterpret_cast<int*>(full + 1);   // [0] next block, [1] its input landed
    const int tid = int(threadIdx.x);
    // The last warp has no x-pass or z-pass line: its lane 0 claims the next
    // block during the x pass (the counter's round trip off the critical
    // path) and fetches its rows; its lanes 0 .. H-1 each store one plane per
    // region (own bulk groups) while the other warps compute.
    constexpr int CLAIMER = cube_threads<S>() - 32;
    static_assert(2 * NP <= CLAIMER && PP <= CLAIMER && H <= 32, "the last warp has no x-pass or z-pass line");
    const bool storer = tid >= CLAIMER && tid < CLAIMER + H;
    const int sp = tid - CLAIMER;   // plane of a storer
    auto claim = [&] { sh[0] = atomicAdd(ctr, 1); };
    auto load = [&] {
        const int t = sh[0];
        if (t < n_items) {
            mbar_expect_tx(full, NL * ROWB);
            tma_2d(reinterpret_cast<void*>(xa), &in_map, 0, items[t].src * NL, full);
        }
    };
    // the 16-byte chunk c of row r (the swizzle XORs address bits 4.. with 7..)
    auto xrow = [&](int r, int c) {
        return *reinterpret_cast<const float4*>(X + r * ROWB + 16u * (unsigned(c) ^ ((unsigned(r) * ROWB >> 7) & SWZ)));
    };
    if (tid == 0) {
        mbar_init(full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == CLAIMER) {
        claim();
        load();
    }
    __syncthreads();
    for (int k = 0;; ++k) {
        const int t = sh[0];
        if (t >= n_items) break;
        const unsigned par = unsigned(k & 1);
        cx<float>* Rg = P + (k & 1) * (H * PP);         // z-pass input, then odd kz
        cx<float>* Eg = P + ((k & 1) ^ 1) * (H * PP);   // even kz
        if (tid == 0) {
            const bool okw = mbar_wait(full, par);
            if (!okw) atomicExch(err, 1);
            sh[1] = okw;
        }
        __syncthreads();
        if (!sh[1]) break;
        mbar_wait(full, par);   // complete: this thread's view of the copies
        // x pass: rows p and p + NP as one complex line, class h = kx parity
        if (tid < 2 * NP) {
            const int h = tid / NP, p = tid % NP;
            cx<float> z[H], o[H];
#pragma unroll
            for (int x = 0; x < NIN; x += 4) {
                const float4 a = xrow(p, x / 4);
                const float4 b = xrow(p + NP, x / 4);
                z[x] = {a.x, b.x};
                z[x + 1] = {a.y, b.y};
                z[x + 2] = {a.z, b.z};
                z[x + 3] = {a.w, b.w};
            }
            cx<float>* d0 = XB + p * RP;
            cx<float>* d1 = XB + (p + NP) * RP;
            // X[kx] and X[S - kx] share a class; split the two real rows
            auto split = [&](int kx, const cx<float>& a, const cx<float>& b) {
                d0[kx] = {0.5f * (a.x + b.x), 0.5f * (a.y - b.y)};
                d1[kx] = {0.5f * (a.y + b.y), 0.5f * (b.x - a.x)};
            };
            if (h == 0) {
                dft_class<S, 2, 0, -1>(z, o);
#pragma unroll
                for (int m = 0; m <= S / 4; ++m) split(2 * m, o[m], o[m == 0 ? 0 : H - m]);
            } else {
                dft_class<S, 2, 1, -1>(z, o);
#pragma unroll
                for (int m = 0; m < S / 4; ++m) split(2 * m + 1, o[m], o[H - 1 - m]);
            }
        }
        if (tid == CLAIMER) claim();
        if (storer) bulk_wait_read<1>();   // the region of the previous even kz is stored
        __syncthreads();
        if (tid == CLAIMER) {
            fence_async_smem();
            load();   // X is free
        }
        // y pass: lines (kx, z), class h = ky parity (whole warps), into planes z of Rg
        if (tid % YC < NX * NIN) {
            const int h = tid / YC, l = tid % YC, kx = l % NX, zz = l / NX;
            cx<float> v[H], o[H];
#pragma unroll
            for (int y = 0; y < H; ++y) v[y] = XB[(zz * NIN + y) * RP + kx];
            if (h == 0) dft_class<S, 2, 0, -1>(v, o);
            else dft_class<S, 2, 1, -1>(v, o);
            cx<float>* col = Rg + zz * PP + kx;
#pragma unroll
            for (int m = 0; m < H; ++m) col[(2 * m + h) * NX] = o[m];
        }
        if (storer) bulk_wait_read<0>();   // the region of the previous odd kz is stored
        __syncthreads();
        cx<float>* out = spec + int64_t(items[t].dst) * NWS;
        // z pass, even kz = 2m into plane m of Eg
        for (int l = tid; l < PP; l += blockDim.x) {
            cx<float> v[H], o[H];
#pragma unroll
            for (int zz = 0; zz < H; ++zz) v[zz] = Rg[zz * PP + l];
            dft_class<S, 2, 0, -1>(v, o);
#pragma unroll
            for (int m = 0; m < H; ++m) Eg[m * PP + l] = o[m];
        }
        fence_async_smem();
        __syncthreads();
        if (storer) {
            bulk_s2g(out + 2 * sp * PP, Eg + sp * PP, PLANE);
            bulk_commit();
        }
        // odd kz = 2m + 1, in place over the line's own column of Rg
        for (int l = tid; l < PP; l += blockDim.x) {
            cx<float> v[H], o[H];
#pragma unroll
            for (int zz = 0; zz < H; ++zz) v[zz] = Rg[zz * PP + l];
            dft_class<S, 2, 1, -1>(v, o);
#pragma unroll
            for (int m = 0; m < H; ++m) Rg[m * PP + l] = o[m];
        }
        fence_async_smem();
        __syncthreads();
        if (storer) {
            bulk_s2g(out + (2 * sp + 1) * PP, Rg + sp * PP, PLANE);
            bulk_commit();
        }
    }
    if (storer) bulk_wait_all();
    __syncthreads();
    if (tid == 0) cube_done(ctr);
}

template <int S, int NOUT>
__global__ void __launch_bounds__(cube_threads<S>(), 1)
    k_c2r_cube(const cx<float>* __restrict__ spec, const C2RItem* __restrict__ items, int n_items,
               float* __restrict__ dst, int64_t dst_stride, const float* __restrict__ add, int add_n,
               int64_t add_stride, int* __restrict__ ctr, int* __restrict__ err) {
    constexpr int NX = S / 2 + 1, PP = S * NX, NL = NOUT * NOUT, NP = NL / 2, N3 = NOUT * NOUT * NOUT;
    constexpr int RP = NX | 1, RS = NOUT | 1, YC = cube_ycls<S>();
    constexpr int64_t NWS = (int64_t(PP) * S + 31) / 32 * 32;
    constexpr unsigned PLANE = PP * unsigned(sizeof(cx<float>));
    static_assert(NOUT == S / 2 && S % 8 == 0 && PP % 2 == 0, "bulk copies move 16-byte multiples");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    cx<float>* B = reinterpret_cast<cx<float>*>(smem_raw);   // S planes
    cx<float>* YB = B + S * PP;                               // [NL rows (z, y)][RP]
    float* O = reinterpret_cast<float*>(YB + NL * RP);        // [NL rows][RS]
    uint64_t* bar = reinterpret_cast<uint64_t*>(O + NL * RS);   // [0] planes < NOUT, [1] the rest
    int* sh = reinterpret_cast<int*>(bar + 2);                 // [0] next block, [1] its input landed
    const int tid = int(threadIdx.x);
    // the last warp, idle in the z pass, claims the next block then
    constexpr int CLAIMER = cube_threads<S>() - 32;
    static_assert(PP <= CLAIMER, "the claiming warp has no z-pass line");
    auto load_lo = [&](int t) {
        mbar_expect_tx(&bar[0], NOUT * PLANE);
        bulk_g2s(B, spec + int64_t(items[t].src) * NWS, NOUT * PLANE, &bar[0]);
    };
    auto load_hi = [&](int t) {
        mbar_expect_tx(&bar[1], (S - NOUT) * PLANE);
        bulk_g2s(B + NOUT * PP, spec + int64_t(items[t].src) * NWS + NOUT * PP, (S - NOUT) * PLANE, &bar[1]);
    };
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == CLAIMER) {
        const int t = atomicAdd(ctr, 1);
        sh[0] = t;
        if (t < n_items) {
            load_lo(t);
            load_hi(t);
        }
    }
    __syncthreads();
    for (int k = 0;; ++k) {
        const int t = sh[0];
        if (t >= n_items) break;
        const unsigned par = unsigned(k & 1);
        if (tid == 0) {
            const bool okw = mbar_wait(&bar[0], par) && mbar_wait(&bar[1], par);
            if (!okw) atomicExch(err, 1);
            sh[1] = okw;
        }
        __syncthreads();
        if (!sh[1]) break;
        mbar_wait(&bar[0], par);   // complete: this thread's view of the copies
        mbar_wait(&bar[1], par);
        // z pass: lines (kx, ky), in place over their own column; keep z < NOUT
        for (int l = tid; l < PP; l += blockDim.x) {
            cx<float>* col = B + l;
            cx<float> v[S];
#pragma unroll
            for (int kz = 0; kz < S; ++kz) v[kz] = col[kz * PP];
            fft<S, S, 1, S>(v);
#pragma unroll
            for (int zz = 0; zz < NOUT; ++zz) col[zz * PP] = v[zz];
        }
        if (tid == CLAIMER) sh[0] = atomicAdd(ctr, 1);
        __syncthreads();
        // planes NOUT and up are free: the next block's arrive meanwhile
        const int tn = sh[0];
        if (tid == CLAIMER && tn < n_items) {
            fence_async_smem();
            load_hi(tn);
        }
        // y pass: lines (kx, z < NOUT), class h = y parity (whole warps), into the row buffer
        if (tid % YC < NX * NOUT) {
            const int h = tid / YC, l = tid % YC, kx = l % NX, zz = l / NX;
            const cx<float>* col = B + zz * PP + kx;
            cx<float> v[S], o[S / 2];
#pragma unroll
            for (int y = 0; y < S; ++y) v[y] = col[y * NX];
            if (h == 0) dft_class<S, 2, 0, 1>(v, o);
            else dft_class<S, 2, 1, 1>(v, o);
#pragma unroll
            for (int m = 0; m < NOUT / 2; ++m) YB[(zz * NOUT + 2 * m + h) * RP + kx] = o[m];
        }
        __syncthreads();
        // planes below NOUT are free too
        if (tid == CLAIMER && tn < n_items) {
            fence_async_smem();
            load_lo(tn);
        }
        // x pass: two Hermitian half-rows (rows p and p + NP) per complex
        // inverse, class r = x mod 4
        if (tid < 4 * NP) {
            const int r = tid / NP, p = tid % NP;
            const cx<float>* a = YB + p * RP;
            const cx<float>* b = YB + (p + NP) * RP;
            cx<float> z[S], o[S / 4];
#pragma unroll
            for (int kx = 0; kx < NX; ++kx) {
                cx<float> A = a[kx], Bk = b[kx];
                if (kx == 0 || 2 * kx == S) {   // exactly real for a real signal
                    A.y = 0.f;
                    Bk.y = 0.f;
                }
                z[kx] = {A.x - Bk.y, A.y + Bk.x};
                if (kx > 0 && S - kx >= NX) z[S - kx] = {A.x + Bk.y, Bk.x - A.y};
            }
            switch (r) {
                case 0: dft_class<S, 4, 0, 1>(z, o); break;
                case 1: dft_class<S, 4, 1, 1>(z, o); break;
                case 2: dft_class<S, 4, 2, 1>(z, o); break;
                default: dft_class<S, 4, 3, 1>(z, o); break;
            }
#pragma unroll
            for (int m = 0; m < NOUT / 4; ++m) {
                O[p * RS + 4 * m + r] = o[m].x;
                O[(p + NP) * RS + 4 * m + r] = o[m].y;
            }
        }
        __syncthreads();
        const C2RItem it = items[t];
        float* out = dst + int64_t(it.dst) * dst_stride;
        const float* ad = (add != nullptr && it.aux >= 0) ? add + int64_t(it.aux) * add_stride : nullptr;
        if (NOUT % 4 == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
            for (int i = tid; i < N3 / 4; i += blockDim.x) {
                const int x = (4 * i) % NOUT, yz = (4 * i) / NOUT;
                float v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = O[yz * RS + x + j];
                if (ad) {
                    const float* q = ad + ((yz / NOUT) * add_n + yz % NOUT) * add_n + x;
#pragma unroll
                    for (int j = 0; j < 4; ++j) v[j] += q[j];
                }
                reinterpret_cast<float4*>(out)[i] = make_float4(v[0], v[1], v[2], v[3]);
            }
        } else {
            for (int i = tid; i < N3; i += blockDim.x) {
                const int x = i % NOUT, yz = i / NOUT;
                float v = O[yz * RS + x];
                if (ad) v += ad[((yz / NOUT) * add_n + yz % NOUT) * add_n + x];
                out[i] = v;
            }
        }
    }
    if (tid == 0) cube_done(ctr);
}

// ---------------------------------------------------------------------------
// Reg (Eq. alg_reg) and Interp (Eq. alg_interp): tensor products of the 1D
// matrices W[c][i][p] (weight of parent node p for child node i).  The two
// n_I x n_I matrices travel as a by-value kernel parameter, so with every loop
// unrolled each weight is a constant-bank operand of an FMA.  One thread holds
// one line of n_I values in registers and produces the n_I outputs of that
// line; the three axes are three such passes through shared memory.
template <typename T, int NI>
struct InterpW {
    T w[2][NI][NI];
};

// Products over the support of each row only (NMAX > 0; interp_lo/len give
// it at compile time after unrolling): the same FMAs in the same order as the
// dense loops minus those with a zero weight, so the same bits.
template <typename T, int NI, int NMAX, int C>
__device__ __forceinline__ void apply_wt_sp(const InterpW<T, NI>& W, const T (&in)[NI], T (&out)[NI]) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int lo = interp_lo(NI - 1, NMAX, C, i), len = interp_len(NI - 1, NMAX, C, i);
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
            if (k < len) out[lo + k] = fma(W.w[C][i][lo + k], in[i], out[lo + k]);
    }
}
template <typename T, int NI, int NMAX, int C>
__device__ __forceinline__ void apply_w_sp(const InterpW<T, NI>& W, const T (&in)[NI], T (&out)[NI]) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int lo = interp_lo(NI - 1, NMAX, C, i), len = interp_len(NI - 1, NMAX, C, i);
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
            if (k < len) out[i] = fma(W.w[C][i][lo + k], in[lo + k], out[i]);
    }
}

// out[p] = sum_i W[c][i][p] in[i]   (adjoint: child line -> parent line).
// c is uniform over the CTA; each branch is a fully unrolled dense product
// (NMAX = 0) or a product over the rows' supports.
template <typename T, int NI, int NMAX = 0>
__device__ __forceinline__ void apply_wt(const InterpW<T, NI>& W, int c, const T (&in)[NI], T (&out)[NI]) {
#pragma unroll
    for (int p = 0; p < NI; ++p) out[p] = T(0);
    if constexpr (NMAX > 0) {
        if (c == 0) apply_wt_sp<T, NI, NMAX, 0>(W, in, out);
        else apply_wt_sp<T, NI, NMAX, 1>(W, in, out);
        return;
    }
    if (c == 0) {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int p = 0; p < NI; ++p) out[p] = fma(W.w[0][i][p], in[i], out[p]);
    } else {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int p = 0; p < NI; ++p) out[p] = fma(W.w[1][i][p], in[i], out[p]);
    }
}

// out[i] = sum_p W[c][i][p] in[p]   (interpolation: parent line -> child line)
template <typename T, int NI, int NMAX = 0>
__device__ __forceinline__ void apply_w(const InterpW<T, NI>& W, int c, const T (&in)[NI], T (&out)[NI]) {
#pragma unroll
    for (int i = 0; i < NI; ++i) out[i] = T(0);
    if constexpr (NMAX > 0) {
        if (c == 0) apply_w_sp<T, NI, NMAX, 0>(W, in, out);
        else apply_w_sp<T, NI, NMAX, 1>(W, in, out);
        return;
    }
    if (c == 0) {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int p = 0; p < NI; ++p) out[i] = fma(W.w[0][i][p], in[p], out[i]);
    } else {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int p = 0; p < NI; ++p) out[i] = fma(W.w[1][i][p], in[p], out[i]);
    }
}

// Compensated form of the two products above (FP32, interpolation mode
// COMPENSATED).  TwoProduct (an FMA gives the exact error of w * x) and
// TwoSum (Knuth: the exact error of s + p in six additions) are error-free
// transformations; adding every error into e (Ogita, Rump and Oishi's Dot2)
// leaves s + e equal to the dot product summed in twice the working
// precision.  The __f*_rn intrinsics are never contracted or reassociated.
// Zero weights (outside the n_max-node window) are skipped.
__device__ __forceinline__ void acc_comp(float& s, float& e, float w, float x) {
    if (w == 0.f) return;
    const float p = __fmul_rn(w, x);
    const float pe = __fmaf_rn(w, x, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float te = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    e = __fadd_rn(e, __fadd_rn(te, pe));
}
template <int NI, int NMAX, int C>
__device__ __forceinline__ void apply_wt_comp_sp(const InterpW<float, NI>& W, const float (&in)[NI], float (&s)[NI],
                                                 float (&e)[NI]) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int lo = interp_lo(NI - 1, NMAX, C, i), len = interp_len(NI - 1, NMAX, C, i);
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
            if (k < len) acc_comp(s[lo + k], e[lo + k], W.w[C][i][lo + k], in[i]);
    }
}
template <int NI, int NMAX, int C>
__device__ __forceinline__ void apply_w_comp_sp(const InterpW<float, NI>& W, const float (&in)[NI], float (&s)[NI],
                                                float (&e)[NI]) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int lo = interp_lo(NI - 1, NMAX, C, i), len = interp_len(NI - 1, NMAX, C, i);
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
            if (k < len) acc_comp(s[i], e[i], W.w[C][i][lo + k], in[lo + k]);
    }
}
// (s, e)[p] += sum_i W[c][i][p] in[i]
template <int NI, int NMAX = 0>
__device__ __forceinline__ void apply_wt_comp(const InterpW<float, NI>& W, int c, const float (&in)[NI],
                                              float (&s)[NI], float (&e)[NI]) {
    if constexpr (NMAX > 0) {
        if (c == 0) apply_wt_comp_sp<NI, NMAX, 0>(W, in, s, e);
        else apply_wt_comp_sp<NI, NMAX, 1>(W, in, s, e);
        return;
    }
    if (c == 0) {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int p = 0; p < NI; ++p) acc_comp(s[p], e[p], W.w[0][i][p], in[i]);
    } else {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int p = 0; p < NI; ++p) acc_comp(s[p], e[p], W.w[1][i][p], in[i]);
    }
}
// (s, e)[i] += sum_p W[c][i][p] in[p]
template <int NI, int NMAX = 0>
__device__ __forceinline__ void apply_w_comp(const InterpW<float, NI>& W, int c, const float (&in)[NI],
                                             float (&s)[NI], float (&e)[NI]) {
    if constexpr (NMAX > 0) {
        if (c == 0) apply_w_comp_sp<NI, NMAX, 0>(W, in, s, e);
        else apply_w_comp_sp<NI, NMAX, 1>(W, in, s, e);
        return;
    }
    if (c == 0) {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int p = 0; p < NI; ++p) acc_comp(s[i], e[i], W.w[0][i][p], in[p]);
    } else {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int p = 0; p < NI; ++p) acc_comp(s[i], e[i], W.w[1][i][p], in[p]);
    }
}

// One pass of a line: out = sum over the given children of the adjoint (Reg)
// products, plain or compensated.
template <typename T, int NI, bool COMP, int NMAX>
struct LineSum {
    T s[NI], e[NI];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int p = 0; p < NI; ++p) s[p] = e[p] = T(0);
    }
    __device__ __forceinline__ void add_wt(const InterpW<T, NI>& W, int c, const T (&in)[NI]) {
        if constexpr (COMP) {
            apply_wt_comp<NI, NMAX>(W, c, in, s, e);
        } else {
            T o[NI];
            apply_wt<T, NI, NMAX>(W, c, in, o);
#pragma unroll
            for (int p = 0; p < NI; ++p) s[p] += o[p];
        }
    }
    __device__ __forceinline__ void add_w(const InterpW<T, NI>& W, int c, const T (&in)[NI]) {
        if constexpr (COMP) {
            apply_w_comp<NI, NMAX>(W, c, in, s, e);
        } else {
            T o[NI];
            apply_w<T, NI, NMAX>(W, c, in, o);
#pragma unroll
            for (int p = 0; p < NI; ++p) s[p] += o[p];
        }
    }
    __device__ __forceinline__ T get(int p) const {
        if constexpr (COMP) return __fadd_rn(s[p], e[p]);
        else return s[p];
    }
};

constexpr int kLineThreads = 320;   // >= 17*17 lines of a pass

// Reg: one CTA per parent interval; the parent's sources accumulate in the
// registers of the z-pass threads across the 8 children.  A level-1 child is a
// block: its sources occupy nodes [0, n_b)^3 and its last node plane is 0.
// One shared buffer: every pass reads its whole line into registers, then a
// barrier, then writes.
template <typename T, int NI, int NMAX = 0>
__global__ void __launch_bounds__(kLineThreads) k_reg(const T* __restrict__ child_src, int child_is_block,
                                                      const int* __restrict__ child_index,
                                                      const int* __restrict__ parent_slot,
                                                      T* __restrict__ dst, const InterpW<T, NI> W) {
    constexpr int NB = NI - 1, N2 = NI * NI, N3 = NI * NI * NI;
    __shared__ T a[N3];
    const int t = threadIdx.x;
    const bool act = t < N2;
    T acc[NI];
#pragma unroll
    for (int r = 0; r < NI; ++r) acc[r] = T(0);
    for (int c = 0; c < 8; ++c) {
        const int src = child_index[blockIdx.x * 8 + c];
        if (src < 0) continue;                               // uniform over the CTA
        const int cxp = c & 1, cyp = (c >> 1) & 1, czp = c >> 2;
        T in[NI], out[NI];
        // x pass: line (z, y) of the child -> a[z][y][p]
        if (act) {
            const int y = t % NI, z = t / NI;
            if (child_is_block) {
                const T* row = child_src + int64_t(src) * NB * NB * NB + (z * NB + y) * NB;
                const bool live = y < NB && z < NB;
#pragma unroll
                for (int x = 0; x < NI; ++x) in[x] = (live && x < NB) ? row[x] : T(0);
            } else {
                const T* row = child_src + int64_t(src) * N3 + (z * NI + y) * NI;
#pragma unroll
                for (int x = 0; x < NI; ++x) in[x] = row[x];
            }
            apply_wt<T, NI, NMAX>(W, cxp, in, out);
        }
        __syncthreads();                                      // previous child's z pass is done with a
        if (act) {
#pragma unroll
            for (int p = 0; p < NI; ++p) a[t * NI + p] = out[p];
        }
        __syncthreads();
        // y pass: line (z, p) -> a[z][q][p]
        if (act) {
            const int p = t % NI, z = t / NI;
#pragma unroll
            for (int y = 0; y < NI; ++y) in[y] = a[(z * NI + y) * NI + p];
            apply_wt<T, NI, NMAX>(W, cyp, in, out);
        }
        __syncthreads();
        if (act) {
            const int p = t % NI, z = t / NI;
#pragma unroll
            for (int q = 0; q < NI; ++q) a[(z * NI + q) * NI + p] = out[q];
        }
        __syncthreads();
        // z pass: line (q, p) -> acc[r]
        if (act) {
#pragma unroll
            for (int z = 0; z < NI; ++z) in[z] = a[z * N2 + t];
            apply_wt<T, NI, NMAX>(W, czp, in, out);
#pragma unroll
            for (int r = 0; r < NI; ++r) acc[r] += out[r];
        }
    }
    if (act) {
        T* o = dst + int64_t(parent_slot[blockIdx.x]) * N3 + t;
#pragma unroll
        for (int r = 0; r < NI; ++r) o[r * N2] = acc[r];
    }
}

// Reg, wide form (FP32; FP64 keeps k_reg, whose registers it would exceed):
// one CTA of kRegThreads per parent takes all 8 children at once.  z pass first: item (cx, cy, x, y) reads the z lines of its two
// children (cz = 0, 1; coalesced along x) and sums their adjoint products into
// a[cx][cy][pz][y][x]; y pass: item (cx, pz, x) sums the two cy lines into
// b[cx][pz][py][x]; x pass: item (pz, py) sums the two cx lines into the
// parent row, staged through shared memory for coalesced stores.  b and the
// staged rows reuse a's storage (every pass reads into registers, then a
// barrier, then writes; each pass has at most one item per thread where it
// writes in place).
constexpr int kRegThreads = 768;   // >= 2 * 17 * 17 (one y-pass item per thread)

template <typename T, int NI>
__host__ __device__ constexpr size_t reg_wide_smem() { return sizeof(T) * 4 * size_t(NI) * NI * NI; }

template <typename T, int NI, bool COMP = false, int NMAX = 0>
__global__ void __launch_bounds__(kRegThreads) k_reg_wide(const T* __restrict__ child_src, int child_is_block,
                                                          const int* __restrict__ child_index,
                                                          const int* __restrict__ parent_slot,
                                                          T* __restrict__ dst, const InterpW<T, NI> W) {
    constexpr int NB = NI - 1, N2 = NI * NI, N3 = NI * NI * NI;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    T* a = reinterpret_cast<T*>(smem_raw);   // [4][NI][NI][NI] = [cx + 2cy][pz][y][x]
    const int t = threadIdx.x;
    // z pass (4 N2 items, a thread may take two)
    for (int it = t; it < 4 * N2; it += kRegThreads) {
        const int x = it % NI, y = (it / NI) % NI, cxy = it / N2;
        LineSum<T, NI, COMP, NMAX> out;
        out.zero();
#pragma unroll
        for (int cz = 0; cz < 2; ++cz) {
            const int s = __ldg(child_index + blockIdx.x * 8 + cxy + 4 * cz);
            if (s < 0) continue;
            T in[NI];
            if (child_is_block) {
                const bool live = x < NB && y < NB;
                const T* col = child_src + int64_t(s) * NB * NB * NB + y * NB + x;
#pragma unroll
                for (int z = 0; z < NI; ++z) in[z] = (live && z < NB) ? __ldg(col + z * NB * NB) : T(0);
            } else {
                const T* col = child_src + int64_t(s) * N3 + y * NI + x;
#pragma unroll
                for (int z = 0; z < NI; ++z) in[z] = __ldg(col + z * N2);
            }
            out.add_wt(W, cz, in);
        }
#pragma unroll
        for (int p = 0; p < NI; ++p) a[(cxy * NI + p) * N2 + y * NI + x] = out.get(p);
    }
    __syncthreads();
    // y pass: 2 N2 items (cx, pz, x) <= kRegThreads, b[cx][pz][py][x] over a
    LineSum<T, NI, COMP, NMAX> yout;
    const bool ya = t < 2 * N2;
    if (ya) {
        const int x = t % NI, pz = (t / NI) % NI, cx = t / N2;
        yout.zero();
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
            T in[NI];
            const T* col = a + ((cx + 2 * cy) * NI + pz) * N2 + x;
#pragma unroll
            for (int y = 0; y < NI; ++y) in[y] = col[y * NI];
            yout.add_wt(W, cy, in);
        }
    }
    __syncthreads();
    if (ya) {
        const int x = t % NI, pz = (t / NI) % NI, cx = t / N2;
#pragma unroll
        for (int p = 0; p < NI; ++p) a[((cx * NI + pz) * NI + p) * NI + x] = yout.get(p);
    }
    __syncthreads();
    // x pass: N2 items (pz, py); rows staged in a, then stored coalesced
    LineSum<T, NI, COMP, NMAX> xout;
    const bool xa = t < N2;
    if (xa) {
        const int py = t % NI, pz = t / NI;
        xout.zero();
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
            T in[NI];
            const T* row = a + ((cx * NI + pz) * NI + py) * NI;
#pragma unroll
            for (int x = 0; x < NI; ++x) in[x] = row[x];
            xout.add_wt(W, cx, in);
        }
    }
    __syncthreads();
    if (xa) {
#pragma unroll
        for (int p = 0; p < NI; ++p) a[t * NI + p] = xout.get(p);
    }
    __syncthreads();
    T* o = dst + int64_t(__ldg(parent_slot + blockIdx.x)) * N3;
    for (int i = t; i < N3; i += kRegThreads) o[i] = a[i];
}

// Interp: u[slot] += (W_cz x W_cy x W_cx) up[parent], c = slot & 7.
// With block != nullptr the output is the child's first NI-1 nodes per axis,
// added into u at block[i] * (NI-1)^3 (a level-1 interval's block points).
template <typename T, int NI, bool COMP = false, int NMAX = 0>
__global__ void __launch_bounds__(kLineThreads) k_interp(const int* __restrict__ slot,
                                                         const int* __restrict__ parent, T* __restrict__ u,
                                                         const T* __restrict__ up, const InterpW<T, NI> W,
                                                         int accumulate, const int* __restrict__ block) {
    constexpr int N2 = NI * NI, N3 = NI * NI * NI;
    __shared__ T a[N3];
    const int t = threadIdx.x;
    const bool act = t < N2;
    const int s = slot[blockIdx.x];
    const int c = s & 7, cxp = c & 1, cyp = (c >> 1) & 1, czp = c >> 2;
    const T* U = up + int64_t(parent[blockIdx.x]) * N3;
    T in[NI], out[NI];
    // one line through W_c: plain or compensated sums
    auto line = [&](int cc) {
        LineSum<T, NI, COMP, NMAX> sum;
        sum.zero();
        sum.add_w(W, cc, in);
#pragma unroll
        for (int i = 0; i < NI; ++i) out[i] = sum.get(i);
    };
    // x pass: line (pz, py) -> a[pz][py][ix]
    if (act) {
#pragma unroll
        for (int x = 0; x < NI; ++x) in[x] = U[t * NI + x];
        line(cxp);
#pragma unroll
        for (int x = 0; x < NI; ++x) a[t * NI + x] = out[x];
    }
    __syncthreads();
    // y pass: line (pz, ix) -> a[pz][iy][ix]
    if (act) {
        const int ix = t % NI, z = t / NI;
#pragma unroll
        for (int y = 0; y < NI; ++y) in[y] = a[(z * NI + y) * NI + ix];
        line(cyp);
    }
    __syncthreads();
    if (act) {
        const int ix = t % NI, z = t / NI;
#pragma unroll
        for (int y = 0; y < NI; ++y) a[(z * NI + y) * NI + ix] = out[y];
    }
    __syncthreads();
    // z pass: line (iy, ix) -> u[iz][iy][ix] +=
    if (act) {
#pragma unroll
        for (int z = 0; z < NI; ++z) in[z] = a[z * N2 + t];
        line(czp);
        if (block) {
            constexpr int NB = NI - 1;
            const int ix = t % NI, iy = t / NI;
            if (ix < NB && iy < NB) {
                T* o = u + int64_t(__ldg(block + blockIdx.x)) * NB * NB * NB + iy * NB + ix;
#pragma unroll
                for (int z = 0; z < NB; ++z) o[z * NB * NB] += out[z];
            }
            return;
        }
        T* o = u + int64_t(s) * N3 + t;
        if (accumulate) {
#pragma unroll
            for (int z = 0; z < NI; ++z) o[z * N2] += out[z];
        } else {
#pragma unroll
            for (int z = 0; z < NI; ++z) o[z * N2] = out[z];
        }
    }
}

}  // namespace dev

// ---------------------------------------------------------------------------
// Launchers

template <typename T, int S, int NIN>
static cudaError_t launch_r2c(const T* src, int64_t stride, const R2CItem* items, int n,
                              void* spec, cudaStream_t st) {
    const size_t smem = dev::fft_smem_bytes<T, S, NIN>();
    auto k = dev::k_r2c<T, S, NIN>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    constexpr int K = dev::fft_items_per_cta<T, S, NIN>();
    k<<<(n + K - 1) / K, dev::fft_threads<T, S, NIN>(), smem, st>>>(src, stride, items,
                                                                     static_cast<dev::cx<T>*>(spec), n);
    return cudaGetLastError();
}

template <typename T, int S, int NOUT>
static cudaError_t launch_c2r(const void* spec, const C2RItem* items, int n, T* dst, int64_t ds,
                              const T* add, int add_n, int64_t as, cudaStream_t st) {
    const size_t smem = dev::fft_smem_bytes<T, S, NOUT>();
    auto k = dev::k_c2r<T, S, NOUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    constexpr int K = dev::fft_items_per_cta<T, S, NOUT>();
    k<<<(n + K - 1) / K, dev::fft_threads<T, S, NOUT>(), smem, st>>>(static_cast<const dev::cx<T>*>(spec), items,
                                                                      dst, ds, add, add_n, as, n);
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
    return LaunchExt<T>::r2c(S, n_in, src, stride, items, n, spec, st);
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
    return LaunchExt<T>::c2r(S, n_out, spec, items, n, dst, ds, add, add_n, as, st);
}

// The near-field products of the separate level-0 form (Sec. 3.1 lists): one
// kernel for every transform length, the spectrum size a run-time argument.
template <typename T>
cudaError_t Launch<T>::mac_level0(const void* fh, const void* kh, void* uh, const int* gnbr, int n_groups,
                                  int S, int variant, cudaStream_t st) {
    (void)variant;
    if (n_groups == 0) return cudaSuccess;
    const int64_t NW = nw_of(S), NWS = nws_of(S);
    dim3 block(32, 8), grid((n_groups + 7) / 8, unsigned((NW + 31) / 32));
    dev::k_mac_level0<T><<<grid, block, 0, st>>>(static_cast<const dev::cx<T>*>(fh),
                                                 static_cast<const dev::cx<T>*>(kh), static_cast<dev::cx<T>*>(uh),
                                                 gnbr, n_groups, NW, NWS);
    return cudaGetLastError();
}

template <typename T, int S>
static cudaError_t launch_mac_interval(const void* fh, const void* kh, void* uh, const int* gnbr, const int* order,
                                       int n_groups, int variant, int include_self, const CUtensorMap* tmap, int* err,
                                       cudaStream_t st, int oct = 0, int gpc = 0) {
    constexpr int64_t NW = int64_t(S / 2 + 1) * S * S;
    const auto* f = static_cast<const dev::cx<T>*>(fh);
    const auto* k = static_cast<const dev::cx<T>*>(kh);
    auto* u = static_cast<dev::cx<T>*>(uh);
    // groups per CTA: at least one per warp, and enough CTAs for ~4 waves;
    // several groups per warp even out uneven neighbour counts
    auto groups_per_cta = [&](int warps, int per_sm, int64_t nchunks) {
        // a caller's choice (the interaction-list chunk of the autotuner):
        // whole warps' worth of groups
        if (gpc > 0) return std::max(warps, (gpc + warps - 1) / warps * warps);
        int per = warps;
        while (per < n_groups && int64_t((n_groups + 2 * per - 1) / (2 * per)) * nchunks >= 4 * per_sm * 152)
            per *= 2;
        return per;
    };
    if (variant == 2) variant = 1;                            // (the two-frequency form was removed)
    if (oct && variant == 3) variant = 1;                     // it stages the half table itself
    if (variant == 3 && sizeof(T) == 4) {
        const size_t smem = sizeof(dev::cx<T>) * 343 * 32;
        auto kern = dev::k_mac_interval_pair<T, S>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        if (n_groups == 0) return cudaSuccess;
        const int64_t nchunks = (NW + 31) / 32;
        int per = groups_per_cta(2 * dev::kMacPWarps, 1, nchunks);
        dim3 block(32, dev::kMacPWarps), grid((n_groups + per - 1) / per, unsigned(nchunks));
        kern<<<grid, block, smem, st>>>(f, k, u, gnbr, order, n_groups, per, include_self);
        return cudaGetLastError();
    }
    // FP32 outside variant 1: packed two-wide FMAs, 8 warps of up to 128
    // registers (two CTAs per SM); variant 1 and FP64: one FMA per real
    // product, 12 warps
    const bool packed = sizeof(T) == 4 && variant != 1;
    const int warps = packed ? dev::kMacPackedWarps : dev::kMacWarps;
    const size_t smem = sizeof(dev::cx<T>) * 343 * 32 + 16;
    auto kern = packed ? dev::k_mac_interval<T, S, dev::kMacPackedWarps, sizeof(T) == 4>
                       : dev::k_mac_interval<T, S, dev::kMacWarps, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    if (n_groups == 0) return cudaSuccess;
    const int64_t nchunks = (NW + 31) / 32;
    const int per = groups_per_cta(warps, sizeof(T) == 4 ? 2 : 1, nchunks);
    dim3 block(32, warps), grid((n_groups + per - 1) / per, unsigned(nchunks));
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    if (tmap) map = *tmap;
    kern<<<grid, block, smem, st>>>(f, k, u, gnbr, order, n_groups, per, include_self, map, tmap && !oct ? 1 : 0, err,
                                    oct);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::mac_interval(const void* fh, const void* kh, void* uh, const int* gnbr, const int* order,
                                    int n_groups, int S, int variant, int include_self, const CUtensorMap* tmap,
                                    int* err, cudaStream_t st, int oct, int gpc) {
#define LGF_MACI(SS)                                                                                            \
    case SS:                                                                                                    \
        return launch_mac_interval<T, SS>(fh, kh, uh, gnbr, order, n_groups, variant, include_self, tmap, err, st, \
                                          oct, gpc);
    switch (S) {
        LGF_MACI(8) LGF_MACI(10) LGF_MACI(16) LGF_MACI(17) LGF_MACI(18) LGF_MACI(32) LGF_MACI(33) LGF_MACI(34)
        LGF_MACI(36)
        default:
            return LaunchExt<T>::mac_interval(fh, kh, uh, gnbr, order, n_groups, S, variant, include_self, tmap, err,
                                              st, oct, gpc);
    }
#undef LGF_MACI
}

// early: programmatic serialization behind the kernel just launched on st
// (the level-0 forward FFT), so the CTAs stage their first coefficient chunks
// while that grid drains
template <int S, int WARPS, bool PACKED>
static cudaError_t launch_mac_persist(const void* fh, const void* kh, void* uh, const PersistPlan& pp, int early,
                                      cudaStream_t st) {
    auto kern = dev::k_mac_persist<S, WARPS, PACKED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dev::kPersistSmem));
    if (e != cudaSuccess) return e;
    if (pp.n_groups == 0 || pp.n_cta == 0) return cudaSuccess;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    if (pp.tmap) map = *pp.tmap;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(pp.n_cta));
    cfg.blockDim = dim3(32u * WARPS);
    cfg.dynamicSmemBytes = dev::kPersistSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = early ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<const dev::cx<float>*>(fh),
                              static_cast<const dev::cx<float>*>(kh), static_cast<dev::cx<float>*>(uh), pp.pairs,
                              pp.start, pp.order, pp.cta_units, pp.n_groups, pp.err, map, pp.tmap ? 1 : 0);
}

template <int S>
static cudaError_t launch_mac_persist_form(const void* fh, const void* kh, void* uh, const PersistPlan& pp, int early,
                                           cudaStream_t st) {
    if (pp.packed) return launch_mac_persist<S, dev::kPersistWarpsPacked, true>(fh, kh, uh, pp, early, st);
    return launch_mac_persist<S, dev::kPersistWarps, false>(fh, kh, uh, pp, early, st);
}

template <typename T>
cudaError_t Launch<T>::mac_persist(const void* fh, const void* kh, void* uh, const PersistPlan& pp, int S,
                                   int early, cudaStream_t st) {
    if constexpr (sizeof(T) != 4) {
        return cudaErrorInvalidValue;
    } else {
#define LGF_MACP(SS) \
    case SS: return launch_mac_persist_form<SS>(fh, kh, uh, pp, early, st);
        switch (S) {
            LGF_MACP(8) LGF_MACP(10) LGF_MACP(16) LGF_MACP(17) LGF_MACP(18) LGF_MACP(32) LGF_MACP(33) LGF_MACP(34)
            LGF_MACP(36)
            default: return LaunchExt<T>::mac_persist(fh, kh, uh, pp, S, early, st);
        }
#undef LGF_MACP
    }
}

template <typename T, int NI>
static dev::InterpW<T, NI> pack_w(const T* W) {
    dev::InterpW<T, NI> p;
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < NI; ++i)
            for (int q = 0; q < NI; ++q) p.w[c][i][q] = W[(c * NI + i) * NI + q];
    return p;
}

template <typename T, int NI, int NMAX>
static cudaError_t launch_reg(const T* child_src, int child_is_block, const int* child_index, const int* parent_slot,
                              int n_parents, T* dst, const T* W, int comp, cudaStream_t st) {
    if constexpr (sizeof(T) == 8) {
        dev::k_reg<T, NI, NMAX><<<n_parents, dev::kLineThreads, 0, st>>>(child_src, child_is_block, child_index,
                                                                        parent_slot, dst, pack_w<T, NI>(W));
        return cudaGetLastError();
    } else {
        constexpr size_t smem = dev::reg_wide_smem<T, NI>();
        auto kern = comp ? dev::k_reg_wide<T, NI, true, NMAX> : dev::k_reg_wide<T, NI, false, NMAX>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        kern<<<n_parents, dev::kRegThreads, smem, st>>>(child_src, child_is_block, child_index, parent_slot, dst,
                                                        pack_w<T, NI>(W));
        return cudaGetLastError();
    }
}

// W here is the host copy of the 2 x n_I x n_I matrices (plan precision).
// Stencils with a supported n_max run over each row's support only.
template <typename T>
cudaError_t Launch<T>::reg(int n_b, int n_max, const T* child_src, int child_is_block,
                           const int* child_index, const int* parent_slot, int n_parents, T* dst,
                           const T* W, int comp, cudaStream_t st) {
    if (n_parents == 0) return cudaSuccess;
    const int nm = interp_sparse(n_b, n_max) ? n_max : 0;
#define LGF_REG(NI, NM)                                                                                       \
    if (n_b + 1 == NI && nm == NM)                                                                            \
        return launch_reg<T, NI, NM>(child_src, child_is_block, child_index, parent_slot, n_parents, dst, W, comp, st);
    LGF_REG(5, 0) LGF_REG(9, 0) LGF_REG(9, 7) LGF_REG(9, 9) LGF_REG(17, 0) LGF_REG(17, 7) LGF_REG(17, 9)
#undef LGF_REG
    return LaunchExt<T>::reg(n_b, n_max, child_src, child_is_block, child_index, parent_slot, n_parents, dst, W, comp,
                             st);
}

template <typename T>
cudaError_t Launch<T>::interp(int n_b, int n_max, const int* slot, const int* parent, int n_items, T* u,
                              const T* up, const T* W, int accumulate, const int* block, int comp,
                              cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const int nm = interp_sparse(n_b, n_max) ? n_max : 0;
#define LGF_INTERP(NI, NM)                                                                                    \
    if (n_b + 1 == NI && nm == NM) {                                                                          \
        auto kern = comp ? dev::k_interp<T, NI, sizeof(T) == 4, NM> : dev::k_interp<T, NI, false, NM>;          \
        kern<<<n_items, dev::kLineThreads, 0, st>>>(slot, parent, u, up, pack_w<T, NI>(W), accumulate, block); \
        return cudaGetLastError();                                                                            \
    }
    LGF_INTERP(5, 0) LGF_INTERP(9, 0) LGF_INTERP(9, 7) LGF_INTERP(9, 9) LGF_INTERP(17, 0) LGF_INTERP(17, 7)
    LGF_INTERP(17, 9)
#undef LGF_INTERP
    return LaunchExt<T>::interp(n_b, n_max, slot, parent, n_items, u, up, W, accumulate, block, comp, st);
}

}  // namespace lgf
