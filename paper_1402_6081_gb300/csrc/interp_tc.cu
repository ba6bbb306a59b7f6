// Reg (Eq. alg_reg) and Interp (Eq. alg_interp) on the tensor cores, for FP32
// plans created with a reduced-precision interpolation mode: each axis pass
// of the tensor-product contraction is a GEMM
//     D[line][n] = sum_k A[line][k] B[n][k]
// over the n_I^2 lines of an interval (M tiles of 128 lines), with K = N = n_I
// padded to 16 or 32, issued as tcgen05.mma kind::f16 (BF16 or FP16 inputs,
// FP32 accumulation in tensor memory).  The field between passes stays in FP32
// in shared memory; only the MMA inputs are rounded:
//   LGF_INTERP_BF16    one BF16 product
//   LGF_INTERP_FP16    one FP16 product
//   LGF_INTERP_BF16X3  x and w split into three BF16 parts each
//                      (x = a1 + a2 + a3 exactly up to the last part's
//                      rounding), six products a_i w_j with i + j <= 4:
//                      close to FP32 accuracy
// Operands are K-major without swizzle: 8-row x 16-byte core matrices, the
// rows of a K chunk of 8 contiguous (stride 128 bytes per 8 rows), K chunks
// LBO bytes apart.  One thread issues the MMAs and commits them to an
// mbarrier; every wait is bounded and sets the plan's error flag when it runs
// out; the CTA always frees its tensor memory before it returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lgf_internal.h"

namespace lgf {
namespace tc {

constexpr int kThreads = 384;   // 12 warps: warp w drains tile w / 4, TMEM lanes 32 (w % 4) ..

template <int NI>
struct Shape {
    static constexpr int KP = NI <= 16 ? 16 : 32;   // K and N, padded
    static constexpr int N2 = NI * NI, N3 = NI * NI * NI;
    static constexpr int TILES = (N2 + 127) / 128;
    static constexpr int ROWS = TILES * 128;
    static constexpr uint32_t A_LBO = ROWS / 8 * 128;   // bytes between K chunks of A
    static constexpr uint32_t A_BYTES = uint32_t(ROWS) * KP * 2;
    static constexpr uint32_t B_LBO = KP / 8 * 128;
    static constexpr uint32_t B_BYTES = uint32_t(KP) * KP * 2;
    static constexpr uint32_t COLS = TILES * KP;   // tensor-memory columns of one D
};

template <int NI>
struct Weights {
    float w[2][NI][NI];   // w[c][i][p]: weight of parent node p for child node i
};

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo) {
    uint64_t d = uint64_t((addr >> 4) & 0x3FFF);
    d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((128u >> 4) & 0x3FFF) << 32;   // 8-row groups 128 bytes apart
    d |= uint64_t(1) << 46;                      // tcgen05 descriptor version; no swizzle
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, A and B of one type
// (0 = FP16, 1 = BF16), both K-major, N and M
template <int MODE, int N>
__host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | (uint32_t(MODE == 2 ? 0 : 1) << 7) | (uint32_t(MODE == 2 ? 0 : 1) << 10) |
           (uint32_t(N >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

template <int MODE>
struct Parts {
    static constexpr int P = MODE == 3 ? 3 : 1;
    static constexpr int NPROD = MODE == 3 ? 6 : 1;
};

// bits of the p-th part of x in the mode's input type
template <int MODE>
__device__ __forceinline__ void split(float x, uint16_t (&o)[Parts<MODE>::P]) {
    if constexpr (MODE == 2) {
        o[0] = __half_as_ushort(__float2half_rn(x));
    } else if constexpr (MODE == 1) {
        o[0] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
    } else {
        const __nv_bfloat16 a1 = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(a1);
        const __nv_bfloat16 a2 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(a2);
        o[0] = __bfloat16_as_ushort(a1);
        o[1] = __bfloat16_as_ushort(a2);
        o[2] = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
    }
}

// byte offset of (row, k) in a K-major no-swizzle operand with the given LBO
__device__ __forceinline__ uint32_t kmaj(int row, int k, uint32_t lbo) {
    return uint32_t(k >> 3) * lbo + uint32_t(row >> 3) * 128u + uint32_t(row & 7) * 16u + uint32_t(k & 7) * 2u;
}

__device__ __forceinline__ void mbar_init(uint64_t* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// bounded wait (about 2^31 SM cycles, ~1 s)
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(su32(b)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1LL << 31)) return false;
    }
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}

// 16 or 32 consecutive FP32 columns of this thread's TMEM lane
template <int KP>
__device__ __forceinline__ void tmem_ld(uint32_t addr, float (&v)[KP]) {
    uint32_t r[KP];
    if constexpr (KP == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(addr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
            "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(addr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < KP; ++i) v[i] = __uint_as_float(r[i]);
}

__host__ __device__ constexpr uint32_t pow2_cols(uint32_t c) {
    return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512;
}

// Shared-memory plan of one CTA
template <int MODE, int NI>
struct Smem {
    using S = Shape<NI>;
    static constexpr int P = Parts<MODE>::P;
    static constexpr uint32_t A_OFF = 0;
    static constexpr uint32_t B_OFF = A_OFF + P * S::A_BYTES;              // [2 c][P]
    static constexpr uint32_t X_OFF = B_OFF + 2 * P * S::B_BYTES;          // FP32 field, n_I^3
    static constexpr uint32_t BAR_OFF = (X_OFF + 4 * S::N3 + 15) / 16 * 16;
    static constexpr uint32_t BYTES = BAR_OFF + 16;
};

// The CTA's common state: tensor memory, the barrier, commit count.
struct Ctx {
    uint32_t taddr;
    uint32_t phase;
    uint64_t* bar;
    unsigned char* sm;
};

// A pass's operands are in shared memory: issue the products of every tile
// into D (columns dcol + tile * KP) and wait for them.  acc_in: the first
// product also accumulates into what D holds.
template <int MODE, int NI>
__device__ bool run_pass(Ctx& cx, uint32_t b_off, uint32_t dcol, bool acc_in) {
    using S = Shape<NI>;
    constexpr int NPROD = Parts<MODE>::NPROD;
    // products a_i w_j of the split parts with i + j <= 2 (0-based), in
    // increasing order of size: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = su32(cx.sm + Smem<MODE, NI>::A_OFF), b0 = su32(cx.sm + b_off);
        for (int t = 0; t < S::TILES; ++t) {
            bool first = !acc_in;
            for (int s = 0; s < S::KP / 16; ++s)
                for (int q = 0; q < NPROD; ++q) {
                    const int pa = q == 2 || q == 4 ? 1 : q == 5 ? 2 : 0;
                    const int pb = q == 1 || q == 4 ? 1 : q == 3 ? 2 : 0;
                    const uint64_t ad = smem_desc(a0 + pa * S::A_BYTES + uint32_t(t) * 2048u + s * 2u * S::A_LBO,
                                                  S::A_LBO);
                    const uint64_t bd = smem_desc(b0 + pb * S::B_BYTES + s * 2u * S::B_LBO, S::B_LBO);
                    mma(cx.taddr + dcol + uint32_t(t * S::KP), ad, bd, idesc<MODE, S::KP>(), first ? 0u : 1u);
                    first = false;
                }
        }
        commit(cx.bar);
    }
    const bool ok = mbar_wait(cx.bar, cx.phase & 1);
    cx.phase++;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return __syncthreads_and(ok) != 0;
}

// this thread's D row of the pass (tile w / 4, lane quarter w % 4) into v;
// returns the line index, or -1 when the row is padding or the warp has no tile
template <int NI>
__device__ int drain(const Ctx& cx, uint32_t dcol, float (&v)[Shape<NI>::KP]) {
    using S = Shape<NI>;
    const int w = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    const int tile = w / 4;
    if (tile >= S::TILES) return -1;
    const uint32_t addr = cx.taddr + (uint32_t(32 * (w % 4)) << 16) + dcol + uint32_t(tile * S::KP);
    tmem_ld<S::KP>(addr, v);
    const int row = 128 * tile + 32 * (w % 4) + lane;
    return row < S::N2 ? row : -1;
}

// A of a pass from the FP32 field X: axis 0 lines (z, y) over x, axis 1 lines
// (z, x) over y, axis 2 lines (y, x) over z
template <int MODE, int NI>
__device__ void build_a(unsigned char* sm, const float* X, int axis) {
    using S = Shape<NI>;
    constexpr int P = Parts<MODE>::P;
    for (int i = threadIdx.x; i < S::N3; i += kThreads) {
        const int l = i / NI, k = i % NI;   // line, position along the axis
        const int a = l / NI, b = l % NI;
        const float x = axis == 0 ? X[(a * NI + b) * NI + k] : axis == 1 ? X[(a * NI + k) * NI + b] : X[k * S::N2 + l];
        uint16_t o[P];
        split<MODE>(x, o);
#pragma unroll
        for (int p = 0; p < P; ++p)
            *reinterpret_cast<uint16_t*>(sm + Smem<MODE, NI>::A_OFF + p * S::A_BYTES + kmaj(l, k, S::A_LBO)) = o[p];
    }
}

// B[c][part]: B[n][k] = W[c][n][k] (Interp) or W[c][k][n] (Reg, the adjoint)
template <int MODE, int NI>
__device__ void build_b(unsigned char* sm, const Weights<NI>& W, bool adjoint) {
    using S = Shape<NI>;
    constexpr int P = Parts<MODE>::P;
    for (int i = threadIdx.x; i < 2 * NI * NI; i += kThreads) {
        const int c = i / (NI * NI), n = (i / NI) % NI, k = i % NI;
        uint16_t o[P];
        split<MODE>(adjoint ? W.w[c][k][n] : W.w[c][n][k], o);
#pragma unroll
        for (int p = 0; p < P; ++p)
            *reinterpret_cast<uint16_t*>(sm + Smem<MODE, NI>::B_OFF + (c * P + p) * S::B_BYTES +
                                         kmaj(n, k, S::B_LBO)) = o[p];
    }
}

template <int MODE, int NI>
__device__ void zero_operands(unsigned char* sm) {
    uint32_t* z = reinterpret_cast<uint32_t*>(sm);
    for (uint32_t i = threadIdx.x; i < Smem<MODE, NI>::X_OFF / 4; i += kThreads) z[i] = 0u;
}

template <int MODE, int NI>
__device__ bool setup(Ctx& cx, unsigned char* sm, uint32_t ncols) {
    cx.sm = sm;
    cx.bar = reinterpret_cast<uint64_t*>(sm + Smem<MODE, NI>::BAR_OFF);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + Smem<MODE, NI>::BAR_OFF + 8);
    cx.phase = 0;
    if (threadIdx.x == 0) mbar_init(cx.bar);
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    cx.taddr = *tslot;
    return true;
}

__device__ __forceinline__ void teardown(const Ctx& cx, uint32_t ncols) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(cx.taddr), "r"(ncols) : "memory");
}

// Interp: u[slot] (+)= (W_cz x W_cy x W_cx) up[parent], c = slot & 7; with
// block != nullptr the first n_I - 1 nodes per axis are added into the block.
template <int MODE, int NI>
__global__ void __launch_bounds__(kThreads, 1)
    k_interp_tc(const int* __restrict__ slot, const int* __restrict__ parent, float* __restrict__ u,
                const float* __restrict__ up, const Weights<NI> W, int accumulate, const int* __restrict__ block,
                int* __restrict__ err) {
    using S = Shape<NI>;
    using SM = Smem<MODE, NI>;
    constexpr uint32_t ncols = pow2_cols(S::COLS);
    extern __shared__ __align__(1024) unsigned char sm[];
    float* X = reinterpret_cast<float*>(sm + SM::X_OFF);
    zero_operands<MODE, NI>(sm);
    __syncthreads();
    build_b<MODE, NI>(sm, W, false);
    const int s = __ldg(slot + blockIdx.x);
    const int c = s & 7;
    const float* U = up + int64_t(__ldg(parent + blockIdx.x)) * S::N3;
    for (int i = threadIdx.x; i < S::N3; i += kThreads) X[i] = __ldg(U + i);
    Ctx cx;
    setup<MODE, NI>(cx, sm, ncols);
    bool ok = true;
    for (int axis = 0; axis < 3 && ok; ++axis) {
        build_a<MODE, NI>(sm, X, axis);
        const int cb = (c >> axis) & 1;
        ok = run_pass<MODE, NI>(cx, SM::B_OFF + cb * Parts<MODE>::P * S::B_BYTES, 0, false);
        if (!ok) break;
        float v[S::KP];
        const int row = drain<NI>(cx, 0, v);
        if (row >= 0) {
            const int a = row / NI, b = row % NI;
            if (axis == 0) {
#pragma unroll
                for (int n = 0; n < NI; ++n) X[(a * NI + b) * NI + n] = v[n];
            } else if (axis == 1) {
#pragma unroll
                for (int n = 0; n < NI; ++n) X[(a * NI + n) * NI + b] = v[n];
            } else if (block) {
                constexpr int NB = NI - 1;
                if (a < NB && b < NB) {
                    float* o = u + int64_t(__ldg(block + blockIdx.x)) * NB * NB * NB + a * NB + b;
#pragma unroll
                    for (int n = 0; n < NB; ++n) o[n * NB * NB] += v[n];
                }
            } else {
                float* o = u + int64_t(s) * S::N3 + row;
                if (accumulate) {
#pragma unroll
                    for (int n = 0; n < NI; ++n) o[n * S::N2] += v[n];
                } else {
#pragma unroll
                    for (int n = 0; n < NI; ++n) o[n * S::N2] = v[n];
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    teardown(cx, ncols);
}

// Reg: dst[parent_slot] = sum over the 8 children of (W_czT x W_cyT x W_cxT)
// child; a level-1 child is a block (sources on nodes [0, n_I - 1)^3).  The x
// and y passes of a child go through D0; its z pass accumulates into D1.
template <int MODE, int NI>
__global__ void __launch_bounds__(kThreads, 1)
    k_reg_tc(const float* __restrict__ child_src, int child_is_block, const int* __restrict__ child_index,
             const int* __restrict__ parent_slot, float* __restrict__ dst, const Weights<NI> W,
             int* __restrict__ err) {
    using S = Shape<NI>;
    using SM = Smem<MODE, NI>;
    constexpr int NB = NI - 1;
    constexpr uint32_t ncols = pow2_cols(2 * S::COLS);
    extern __shared__ __align__(1024) unsigned char sm[];
    float* X = reinterpret_cast<float*>(sm + SM::X_OFF);
    zero_operands<MODE, NI>(sm);
    __syncthreads();
    build_b<MODE, NI>(sm, W, true);
    Ctx cx;
    setup<MODE, NI>(cx, sm, ncols);
    bool ok = true, any = false;
    for (int c = 0; c < 8 && ok; ++c) {
        const int src = __ldg(child_index + blockIdx.x * 8 + c);
        if (src < 0) continue;   // uniform over the CTA
        if (child_is_block) {
            const float* B = child_src + int64_t(src) * NB * NB * NB;
            for (int i = threadIdx.x; i < S::N3; i += kThreads) {
                const int x = i % NI, y = (i / NI) % NI, z = i / S::N2;
                X[i] = (x < NB && y < NB && z < NB) ? __ldg(B + (z * NB + y) * NB + x) : 0.f;
            }
        } else {
            const float* B = child_src + int64_t(src) * S::N3;
            for (int i = threadIdx.x; i < S::N3; i += kThreads) X[i] = __ldg(B + i);
        }
        for (int axis = 0; axis < 3 && ok; ++axis) {
            build_a<MODE, NI>(sm, X, axis);
            const int cb = (c >> axis) & 1;
            const uint32_t boff = SM::B_OFF + cb * Parts<MODE>::P * S::B_BYTES;
            if (axis < 2) {
                ok = run_pass<MODE, NI>(cx, boff, 0, false);
                if (!ok) break;
                float v[S::KP];
                const int row = drain<NI>(cx, 0, v);
                if (row >= 0) {
                    const int a = row / NI, b = row % NI;
                    if (axis == 0) {
#pragma unroll
                        for (int n = 0; n < NI; ++n) X[(a * NI + b) * NI + n] = v[n];
                    } else {
#pragma unroll
                        for (int n = 0; n < NI; ++n) X[(a * NI + n) * NI + b] = v[n];
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
            } else {
                ok = run_pass<MODE, NI>(cx, boff, S::COLS, any);
                any = true;
            }
        }
    }
    if (ok) {
        float v[S::KP];
        const int row = any ? drain<NI>(cx, S::COLS, v) : -1;
        float* o = dst + int64_t(__ldg(parent_slot + blockIdx.x)) * S::N3;
        if (any) {
            if (row >= 0) {
#pragma unroll
                for (int n = 0; n < NI; ++n) o[n * S::N2 + row] = v[n];
            }
        } else {
            for (int i = threadIdx.x; i < S::N3; i += kThreads) o[i] = 0.f;
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    teardown(cx, ncols);
}

template <int NI>
static Weights<NI> pack(const float* W) {
    Weights<NI> p;
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < NI; ++i)
            for (int q = 0; q < NI; ++q) p.w[c][i][q] = W[(c * NI + i) * NI + q];
    return p;
}

template <int MODE, int NI>
static cudaError_t launch_interp(const int* slot, const int* parent, int n, float* u, const float* up,
                                 const float* W, int accumulate, const int* block, int* err, cudaStream_t st) {
    auto kern = k_interp_tc<MODE, NI>;
    constexpr size_t smem = Smem<MODE, NI>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    kern<<<n, kThreads, smem, st>>>(slot, parent, u, up, pack<NI>(W), accumulate, block, err);
    return cudaGetLastError();
}

template <int MODE, int NI>
static cudaError_t launch_reg(const float* child_src, int child_is_block, const int* child_index,
                              const int* parent_slot, int n, float* dst, const float* W, int* err, cudaStream_t st) {
    auto kern = k_reg_tc<MODE, NI>;
    // a CTA holding 256 tensor-memory columns asks for enough shared memory
    // that at most two share an SM (512 columns): allocations never wait
    constexpr size_t need = Smem<MODE, NI>::BYTES;
    constexpr size_t smem = pow2_cols(2 * Shape<NI>::COLS) > 128 && need < 102400 ? 102400 : need;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    kern<<<n, kThreads, smem, st>>>(child_src, child_is_block, child_index, parent_slot, dst, pack<NI>(W), err);
    return cudaGetLastError();
}

}  // namespace tc

cudaError_t interp_tc(int mode, int n_b, const int* slot, const int* parent, int n_items, float* u, const float* up,
                      const float* W, int accumulate, const int* block, int* err, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
#define LGF_ITC(M, NI)                                                                                      \
    if (mode == M && n_b + 1 == NI)                                                                         \
        return tc::launch_interp<M, NI>(slot, parent, n_items, u, up, W, accumulate, block, err, st);
    LGF_ITC(1, 5) LGF_ITC(1, 9) LGF_ITC(1, 17)
    LGF_ITC(2, 5) LGF_ITC(2, 9) LGF_ITC(2, 17)
    LGF_ITC(3, 5) LGF_ITC(3, 9) LGF_ITC(3, 17)
#undef LGF_ITC
    return cudaErrorInvalidValue;
}

cudaError_t reg_tc(int mode, int n_b, const float* child_src, int child_is_block, const int* child_index,
                   const int* parent_slot, int n_parents, float* dst, const float* W, int* err, cudaStream_t st) {
    if (n_parents == 0) return cudaSuccess;
#define LGF_RTC(M, NI)                                                                                          \
    if (mode == M && n_b + 1 == NI)                                                                             \
        return tc::launch_reg<M, NI>(child_src, child_is_block, child_index, parent_slot, n_parents, dst, W, err, \
                                     st);
    LGF_RTC(1, 5) LGF_RTC(1, 9) LGF_RTC(1, 17)
    LGF_RTC(2, 5) LGF_RTC(2, 9) LGF_RTC(2, 17)
    LGF_RTC(3, 5) LGF_RTC(3, 9) LGF_RTC(3, 17)
#undef LGF_RTC
    return cudaErrorInvalidValue;
}

}  // namespace lgf
