// Internal declarations shared by the host plan builder and the CUDA kernels.
#pragma once

#include <array>
#include <complex>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include <cuda.h>   // CUtensorMap (a plain struct; no driver call is linked)
#include <cuda_runtime_api.h>

#include "../../include/lgf.h"

namespace lgf {

// ---- status helpers (thread-local message, see lgf_last_error) ----
lgf_status fail(lgf_status code, const std::string& msg);
lgf_status ok();

// ---- FP64 LGF (green.cpp) ----
void green_sorted(const std::vector<std::array<int, 3>>& trip, std::vector<double>& out);
std::shared_ptr<const std::vector<double>> green_abs_table(int h, int V);

// ---- host FP64 FFT (host_fft.cpp) ----
// In-place complex DFT of length n with sign -1 (forward) or +1 (inverse,
// unnormalised), on a strided sequence.
void fft_inplace(std::complex<double>* x, int n, int stride, int sign);
// count lines at base + c*line_stride, each n elements at stride (n <= 96).
void fft_lines(std::complex<double>* base, int n, int stride, int count, int64_t line_stride,
               int sign);

// ---- kernel spectra (plan.cpp) ----
// Spectrum (NW values, w = (kz*S + ky)*NX + kx, scaled by 1/S^3) of the kernel
// vector k(m) = G(h (m - d n_b)), |m_a| <= n - 1, placed at m mod S; tab is the
// dense |offset| table G(h*(a,b,c)) of edge V + 1.
void kernel_spectrum(int n_b, int n, int h, int S, const int d[3], const double* tab, int V,
                     std::complex<double>* outw);

// per-kernel timing capacity of a plan (0 when timing is off)
int plan_timing_capacity(const lgf_plan_s* plan);

// ---- interpolation stencils (plan.cpp) ----
// W[c][i][p] (2 x n_I x n_I) for child c node i and parent node p.
std::vector<double> interp_weights(int n_b, int n_max);

#if defined(__CUDACC__)
#define LGF_HD __host__ __device__
#else
#define LGF_HD
#endif
// Support of row i of W[c] (Sec. 2.5 stencil): child c node i sits at parent
// coordinate x = c n_b / 2 + i / 2.  An integer x is a parent node (one
// weight, 1); otherwise x = k + 1/2 takes the n_max nodes nearest it, the odd
// extra node on the side of the interval centre n_b / 2 (the lower side at the
// centre), shifted inside [0, n_b].  First node and count; interp_weights
// fills exactly these entries and the kernels sum only over them.
LGF_HD constexpr int interp_lo(int n_b, int n_max, int c, int i) {
    const int twice = c * n_b + i;   // 2x
    if (twice % 2 == 0) return twice / 2;
    const int k = twice / 2;
    const int lo = n_max % 2 == 0 ? k - n_max / 2 + 1 : (twice < n_b ? k - (n_max - 1) / 2 + 1 : k - (n_max - 1) / 2);
    const int top = n_b + 1 - n_max;
    return lo < 0 ? 0 : lo > top ? top : lo;
}
LGF_HD constexpr int interp_len(int n_b, int n_max, int c, int i) { return (c * n_b + i) % 2 == 0 ? 1 : n_max; }
// n_max values with support-only Reg/Interp kernels (others: dense loops)
LGF_HD constexpr bool interp_sparse(int n_b, int n_max) { return (n_b == 8 || n_b == 16) && (n_max == 7 || n_max == 9); }

// ---- FFT sizes ----
// Level 0 pads a block of n_b to S0 = 2 n_b per axis; levels >= 1 pad an
// interval of n_I = n_b + 1 nodes to S_I (>= 2 n_I - 1).  R2C keeps
// NX = S/2 + 1 frequencies along x; a spectrum has NW = NX * S * S entries,
// indexed w = (kz * S + ky) * NX + kx.
inline int s_level0(int n_b) { return 2 * n_b; }
int s_interval(int n_b);
inline int nx_of(int S) { return S / 2 + 1; }
inline int64_t nw_of(int S) { return int64_t(nx_of(S)) * S * S; }
// Stride between consecutive spectra in memory: NW rounded up to 32 entries,
// so every spectrum starts 256-byte aligned (FP32) and vector loads of
// frequency pairs stay aligned whatever the parity of NW.
inline int64_t nws_of(int S) { return (nw_of(S) + 31) / 32 * 32; }

// ---- kernel-side parameter blocks ----
struct R2CItem { int src; int dst; };      // source index -> spectrum slot
struct C2RItem { int src; int dst; int aux; };

// Work lists of the persistent interaction kernel: per group, in work order,
// its source groups with the coefficient row of their centre offset d = 2e
// (row (dx+3) + 7 (dy+3) + 49 (dz+3) of the 7^3 table).  Each CTA takes
// floor(chunks / n_cta) whole frequency chunks and then a range of about
// equal work of the units (chunk * n_groups + position) of the chunks left
// over, so it stages as few chunks as it can; err is set when a wait in the
// kernel runs out.
struct PairSrc { int src; int centre; };
struct PersistPlan {
    const CUtensorMap* tmap = nullptr;   // the level's kernel table as a 2D tensor (rows x 2 NWS reals)
    const PairSrc* pairs = nullptr;
    const int* start = nullptr;          // n_groups + 1 offsets into pairs
    const int* order = nullptr;          // group id per position
    const long long* cta_units = nullptr;    // n_cta x {m0, m1, r0, r1}: whole chunks, then leftover units
    int n_groups = 0, n_cta = 0;
    int* err = nullptr;
    bool packed = false;                 // fma.rn.f32x2 form of the products
};

// Launchers (kernels.cu); T = float or double.  All asynchronous on `stream`.
template <typename T>
struct Launch {
    // Twiddle tables into constant memory of the current device.
    static cudaError_t init_twiddles();
    // R2C of items: input n_in^3 (stride n_in) zero-padded to S^3.
    static cudaError_t r2c(int S, int n_in, const T* src, int64_t src_stride,
                           const R2CItem* items, int n_items, void* spec, cudaStream_t st);
    // C2R of items, truncated to n_out^3, written to dst[item.dst*n_out^3] (+add).
    static cudaError_t c2r(int S, int n_out, const void* spec, const C2RItem* items, int n_items,
                           T* dst, int64_t dst_stride, const T* add, int add_n, int64_t add_stride,
                           cudaStream_t st);
    // variant: 0/2 default form, 1 the earlier form (kept for comparison)
    static cudaError_t mac_level0(const void* fh, const void* kh, void* uh, const int* gnbr,
                                  int n_groups, int S, int variant, cudaStream_t st);
    // order: the groups in work order (descending neighbour count);
    // include_self: the group's own block is a source (merged levels 0 and 1)
    // tmap: the kernel table as a 2D tensor for TMA loads of the coefficient
    // chunk (nullptr: plain loads); err: device flag for a wait that ran out
    // oct: kh is the 40-row reflection-reduced table (Sec. 3.2), gathered per
    // frequency instead of read as the half table; gpc: sibling groups per
    // CTA (the interaction-list chunk; 0 = from the level's size)
    static cudaError_t mac_interval(const void* fh, const void* kh, void* uh, const int* gnbr, const int* order,
                                    int n_groups, int S, int variant, int include_self, const CUtensorMap* tmap,
                                    int* err, cudaStream_t st, int oct = 0, int gpc = 0);
    // The same products as mac_interval from a persistent kernel (one CTA per
    // SM) that stages the coefficient chunks with bulk copies; FP32 only.
    // early: launched with programmatic serialization behind the forward FFT
    // that precedes it on st (the FFT kernel signals its dependents).
    static cudaError_t mac_persist(const void* fh, const void* kh, void* uh, const PersistPlan& pp, int S,
                                   int early, cudaStream_t st);
    // Reg of 8 children into each parent: items (parent slot, child group, child-src kind).
    // comp (FP32): compensated sums (interpolation mode COMPENSATED).
    static cudaError_t reg(int n_b, int n_max, const T* child_src, int child_is_block,
                           const int* child_index, const int* parent_slot, int n_parents,
                           T* dst, const T* W, int comp, cudaStream_t st);
    // u[slot] (+)= Interp(u_parent[parent]) for each item (accumulate: add, else
    // store); with block != nullptr: u[block[i]] += the first n_b nodes per axis.
    static cudaError_t interp(int n_b, int n_max, const int* slot, const int* parent, int n_items,
                              T* u, const T* up, const T* W, int accumulate, const int* block, int comp,
                              cudaStream_t st);
};

// The kernels of the block sizes n_b = 6, 10, 12 and 14 (transform lengths
// 12, 20, 24, 28 at level 0; n_I = 7, 11, 13, 15 at the interval levels),
// compiled in units of their own (kernels_ext_f32.cu, kernels_ext_f64.cu) so
// each unit's build stays short.  Launch<T> hands every size it does not
// have to these; the same arguments and errors (cudaErrorInvalidValue for a
// size neither has).
template <typename T>
struct LaunchExt {
    static cudaError_t init_twiddles();
    static cudaError_t r2c(int S, int n_in, const T* src, int64_t src_stride, const R2CItem* items, int n_items,
                           void* spec, cudaStream_t st);
    static cudaError_t c2r(int S, int n_out, const void* spec, const C2RItem* items, int n_items, T* dst,
                           int64_t dst_stride, const T* add, int add_n, int64_t add_stride, cudaStream_t st);
    static cudaError_t mac_interval(const void* fh, const void* kh, void* uh, const int* gnbr, const int* order,
                                    int n_groups, int S, int variant, int include_self, const CUtensorMap* tmap,
                                    int* err, cudaStream_t st, int oct, int gpc);
    static cudaError_t mac_persist(const void* fh, const void* kh, void* uh, const PersistPlan& pp, int S,
                                   int early, cudaStream_t st);
    static cudaError_t reg(int n_b, int n_max, const T* child_src, int child_is_block, const int* child_index,
                           const int* parent_slot, int n_parents, T* dst, const T* W, int comp, cudaStream_t st);
    static cudaError_t interp(int n_b, int n_max, const int* slot, const int* parent, int n_items, T* u,
                              const T* up, const T* W, int accumulate, const int* block, int comp,
                              cudaStream_t st);
};
// Transform lengths the persistent products kernel is built for (FP32)
bool persist_supported(int S);
// Per-block transforms of the FP32 block sizes 18 and 20 (kernels_fft_large.cu):
// (S, n) = (36, 18), (40, 18..20), (42, 20..21); own twiddle tables
bool fft_large_supported(int S, int n);
cudaError_t fft_large_init_twiddles();
cudaError_t r2c_large(int S, int n_in, const float* src, int64_t stride, const R2CItem* items, int n, void* spec,
                      cudaStream_t st);
cudaError_t c2r_large(int S, int n_out, const void* spec, const C2RItem* items, int n, float* dst, int64_t ds,
                      const float* add, int add_n, int64_t as, cudaStream_t st);
// the even lengths 38..66 of the block sizes 18..32 (kernels_persist_large.cu)
bool persist_large_supported(int S);
cudaError_t mac_persist_large(const void* fh, const void* kh, void* uh, const PersistPlan& pp, int S, int early,
                              cudaStream_t st);

// The steps of a solve with every size a run-time argument (generic.cu), for
// the block sizes without per-size kernels (even n_b of [18, 32]).  The
// transforms pass between the level's spectrum buffer (slot layout) and a
// scratch of n_items x n x S x (S/2 + 1) complex values (n = n_in or n_out),
// with a twiddle table (cos, sin)(2 pi m / S), m < S, in the plan precision;
// Reg and Interp use the 1D matrices W (2 x n_I x n_I, device memory) and a
// scratch of n_ctas x 2 n_I^3 values; Reg also 8 n_parents n_I^3 values of
// slices (one per child).
template <typename T>
struct Generic {
    static cudaError_t r2c(int S, int n_in, const T* src, int64_t src_stride, const R2CItem* items, int n_items,
                           void* spec, void* scratch, const void* twt, cudaStream_t st);
    static cudaError_t c2r(int S, int n_out, const void* spec, const C2RItem* items, int n_items, void* scratch,
                           T* dst, int64_t dst_stride, const T* add, int add_n, int64_t add_stride, const void* twt,
                           cudaStream_t st);
    static cudaError_t mac(const void* fh, const void* kh, void* uh, const int* gnbr, int n_groups, int S,
                           int include_self, cudaStream_t st);
    static cudaError_t reg(int n_b, const T* child_src, int child_is_block, const int* child_index,
                           const int* parent_slot, int n_parents, T* dst, const T* W_dev, int comp, T* scratch,
                           T* slices, int n_ctas, cudaStream_t st);
    static cudaError_t interp(int n_b, const int* slot, const int* parent, int n_items, T* u, const T* up,
                              const T* W_dev, int accumulate, const int* block, int comp, T* scratch, int n_ctas,
                              cudaStream_t st);
};

// Level-0 transforms as persistent kernels, FP32 (kernels_f32.cu): one CTA
// per SM (grid from cube_fft_grid, which also sets the kernels' shared-memory
// limit) takes blocks from the counter pair ctr[0..1] (zero between launches)
// and moves each block's data by bulk copies; the forward transform reads its
// input through in_map (rows of n_in reals, box n_in x n_in^2, swizzle of
// n_in * 4 bytes).  The same transforms as Launch<float>::r2c / c2r.
bool cube_fft_supported(int S, int n);
cudaError_t cube_fft_grid(int S, int n, bool inverse, int n_sm, int* grid);
cudaError_t r2c_cube(int S, int n_in, const CUtensorMap& in_map, const R2CItem* items, int n, void* spec, int grid,
                     int* ctr, int* err, cudaStream_t st);
cudaError_t c2r_cube(int S, int n_out, const void* spec, const C2RItem* items, int n, float* dst, int64_t ds,
                     const float* add, int add_n, int64_t as, int grid, int* ctr, int* err, cudaStream_t st);

// Reg and Interp on the tensor cores for FP32 plans (interp_tc.cu); mode is
// an lgf_interp_mode other than NATIVE, err the plan's device error flag.
cudaError_t interp_tc(int mode, int n_b, const int* slot, const int* parent, int n_items, float* u, const float* up,
                      const float* W, int accumulate, const int* block, int* err, cudaStream_t st);
cudaError_t reg_tc(int mode, int n_b, const float* child_src, int child_is_block, const int* child_index,
                   const int* parent_slot, int n_parents, float* dst, const float* W, int* err, cudaStream_t st);

}  // namespace lgf
