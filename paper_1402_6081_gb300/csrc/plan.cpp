// Host side of the LGF solver: the C ABI, the tree and lists of Sec. 3.1, the
// interpolation stencils of Sec. 2.5, the kernel spectra of Step 0 (Eq.
// precomp), device workspace, and the launch sequence of Steps 1-3.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <type_traits>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "lgf_internal.h"

namespace lgf {

// ---------------------------------------------------------------------------
// status

namespace {
thread_local std::string g_err;
}
lgf_status fail(lgf_status code, const std::string& msg) {
    g_err = msg;
    return code;
}
lgf_status ok() { return LGF_OK; }

static lgf_status cuda_fail(cudaError_t e, const char* where) {
    return fail(LGF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define LGF_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// FFT length along each axis for the interval levels (any S >= 2 n_I - 1 gives
// the same linear convolution; these are the lengths the kernels are built for).
int s_interval(int n_b) {
    switch (n_b) {
        case 4: return 10;
        case 6: return 16;
        case 8: return 18;
        case 10: return 24;
        case 12: return 28;
        case 14: return 32;
        case 16: return 33;
        case 18: return 40;            // 2 n_I + 2 would be 38 = 2 x 19: 40 has the FP32 per-block transform
        default: return 2 * n_b + 2;   // the run-time-size kernels (n_b 20..32; 20 and FP32: per-block)
    }
}
static bool s_interval_supported(int n_b, int S) {
    if (n_b == 8) return S == 17 || S == 18;
    if (n_b == 16) return S == 33 || S == 34 || S == 36;
    return S == s_interval(n_b);
}
// block sizes with per-size kernels (the even sizes 4..16); the other even
// sizes up to 32 run the run-time-size kernels of generic.cu
static bool n_b_specialized(int n_b) { return n_b >= 4 && n_b <= 16 && n_b % 2 == 0; }

// ---------------------------------------------------------------------------
// Interpolation stencil (Sec. 2.5): child c node i sits at parent coordinate
// x = c n_b / 2 + i / 2.  A node on a parent node copies it; otherwise the n_max
// parent nodes nearest x are used (an odd count takes its extra node on the side
// of the interval centre n_b/2, the lower side at the centre), shifted to stay
// inside [0, n_I - 1], with Lagrange weights.

std::vector<double> interp_weights(int n_b, int n_max) {
    const int nI = n_b + 1;
    std::vector<double> W(size_t(2) * nI * nI, 0.0);
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < nI; ++i) {
            const int twice = c * n_b + i;   // 2x
            double* row = &W[(size_t(c) * nI + i) * nI];
            if (twice % 2 == 0) {
                row[twice / 2] = 1.0;
                continue;
            }
            const double x = 0.5 * twice;
            const int lo = interp_lo(n_b, n_max, c, i);
            for (int a = lo; a < lo + n_max; ++a) {
                double w = 1.0;
                for (int b = lo; b < lo + n_max; ++b)
                    if (b != a) w *= (x - b) / double(a - b);
                row[a] = w;
            }
        }
    return W;
}

// ---------------------------------------------------------------------------
// Kernel spectra (Step 0): for offset d = idx(Q) - idx(P) at spacing h, the
// kernel vector k(m) = G(h (m - d n_b)), |m_a| <= n - 1, stored at m mod S and
// transformed by a 3D real FFT in FP64; 1/S^3 of the inverse transform is
// folded in.  Level 0 ("near") keeps the 27 offsets |d| <= 1 with n = n_b;
// interval levels keep all 7^3 offsets |d| <= 3 with n = n_I, zero at the 27
// near ones (those pairs belong to finer levels).

struct SpecEntry {
    int device = 0;
    void* ptr = nullptr;
    size_t bytes = 0;
    // the table as a 2D tensor (rows x 2 NWS reals) for TMA loads of
    // coefficient chunks; valid when has_tmap
    alignas(64) CUtensorMap tmap;
    bool has_tmap = false;
    ~SpecEntry() {
        if (ptr) {
            int cur = 0;
            cudaGetDevice(&cur);
            cudaSetDevice(device);
            cudaFree(ptr);
            cudaSetDevice(cur);
        }
    }
};

struct SpecKey {
    int device, n_b, S, h, near, prec, oct;
    bool operator<(const SpecKey& o) const {
        return std::tie(device, n_b, S, h, near, prec, oct) <
               std::tie(o.device, o.n_b, o.S, o.h, o.near, o.prec, o.oct);
    }
};

void kernel_spectrum(int n_b, int n, int h, int S, const int d[3], const double* tab, int V,
                     std::complex<double>* outw /* NW */) {
    const int NX = nx_of(S);
    std::vector<std::complex<double>> C(size_t(S) * S * NX);
    std::vector<double> k(size_t(S) * S * S, 0.0);
    const size_t Wt = size_t(V) + 1;
    for (int mz = -(n - 1); mz <= n - 1; ++mz)
        for (int my = -(n - 1); my <= n - 1; ++my)
            for (int mx = -(n - 1); mx <= n - 1; ++mx) {
                const int vx = std::abs(mx - d[0] * n_b), vy = std::abs(my - d[1] * n_b),
                          vz = std::abs(mz - d[2] * n_b);
                const int iz = (mz % S + S) % S, iy = (my % S + S) % S, ix = (mx % S + S) % S;
                k[(size_t(iz) * S + iy) * S + ix] = tab[(size_t(vx) * Wt + vy) * Wt + vz];
            }
    (void)h;
    // x: real lines -> first NX frequencies
    std::vector<std::complex<double>> line(S);
    for (int z = 0; z < S; ++z)
        for (int y = 0; y < S; ++y) {
            for (int x = 0; x < S; ++x) line[x] = k[(size_t(z) * S + y) * S + x];
            fft_lines(line.data(), S, 1, 1, 0, -1);
            for (int kx = 0; kx < NX; ++kx) C[(size_t(z) * S + y) * NX + kx] = line[kx];
        }
    // y: lines (z, kx), stride NX; z: lines (y, kx), stride S*NX
    for (int z = 0; z < S; ++z) fft_lines(&C[size_t(z) * S * NX], S, NX, NX, 1, -1);
    fft_lines(C.data(), S, S * NX, S * NX, 1, -1);
    const double inv = 1.0 / (double(S) * S * S);
    for (size_t i = 0; i < C.size(); ++i) outw[i] = C[i] * inv;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); nullptr when unavailable
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// FP32 block inputs (n_blocks blocks of n^3, back to back) as rows of n reals,
// one box per block (n x n^2 rows), 16-byte chunks swizzled within each row
// (the row is 64 bytes for n = 16, 32 for n = 8): the persistent level-0
// forward transform reads it
static bool encode_rows_map(CUtensorMap* m, const float* f, int64_t n_blocks, int n) {
    auto enc = tensor_map_encoder();
    if (!enc || (n != 16 && n != 8) || (reinterpret_cast<uintptr_t>(f) & 15) != 0) return false;
    const cuuint64_t dims[2] = {cuuint64_t(n), cuuint64_t(n_blocks) * cuuint64_t(n) * cuuint64_t(n)};
    const cuuint64_t strides[1] = {cuuint64_t(n) * 4};
    const cuuint32_t box[2] = {cuuint32_t(n), cuuint32_t(n * n)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(f), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE,
                           n == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// rows x NWS complex values viewed as rows x 2 NWS reals; boxes of 32
// complex values (64 reals) by 172 rows (a whole stored half-table chunk)
static bool encode_table_map(SpecEntry& e, int rows, int64_t nws, int prec) {
    auto enc = tensor_map_encoder();
    if (!enc || rows < 172) return false;
    const bool f64 = prec == LGF_FP64;
    const cuuint64_t dims[2] = {cuuint64_t(2 * nws), cuuint64_t(rows)};
    const cuuint64_t strides[1] = {cuuint64_t(2 * nws) * (f64 ? 8 : 4)};
    const cuuint32_t box[2] = {64, 172};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&e.tmap, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, e.ptr,
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static std::mutex g_spec_mu;
static std::map<SpecKey, std::weak_ptr<SpecEntry>> g_spec_cache;

// kind: kNear (27 offsets |d| <= 1, n = n_b), kInterval (343 offsets |d| <= 3,
// n = n_I, zero at the near ones), kBlock (343 offsets |d| <= 3, n = n_b, all
// filled: level 0 near field and level-1 interaction list on the block grid)
enum SpecKind { kNear = 0, kInterval = 1, kBlock = 2 };

// oct (343-offset kinds only): store the 40 representatives of the offsets
// under the reflections of G instead of the 172-row half table (the products
// kernel maps each offset's frequencies onto its representative's)
static lgf_status get_spectra(int device, int n_b, int S, int h, int kind, int prec,
                              std::shared_ptr<SpecEntry>& out, int oct = 0) {
    if (kind == kNear) oct = 0;
    const SpecKey key{device, n_b, S, h, kind, prec, oct};
    std::lock_guard<std::mutex> lock(g_spec_mu);
    auto it = g_spec_cache.find(key);
    if (it != g_spec_cache.end()) {
        if (auto sp = it->second.lock()) {
            out = sp;
            return ok();
        }
    }
    const bool near = kind == kNear;
    const int n = kind == kInterval ? n_b + 1 : n_b;
    const int V = near ? 2 * n_b - 1 : kind == kBlock ? 4 * n_b - 1 : 4 * n_b;
    auto tab = green_abs_table(h, V);
    // The kernel vector of -d is that of d reflected (G is even and the
    // window |m_a| <= n - 1 symmetric), so its spectrum is the complex
    // conjugate: the 343-offset tables keep only the rows id >= 171 (d = 0 and
    // the offsets after it in x-fastest order); row id < 171 is the conjugate
    // of row 342 - id.  The 27-offset table is kept whole.
    const int nd = near ? 27 : oct ? 40 : 172;
    const int first = near ? 0 : 171;
    const int64_t NW = nw_of(S), NWS = nws_of(S);
    std::vector<std::complex<double>> all(size_t(nd) * NWS, 0.0);
    // offset of a stored row: the 27- or 343-offset id, or the representative
    // (|dx|, a, b), a <= b, of the reduced table (row 10 |dx| + b (b + 1) / 2 + a)
    auto offset_of = [&](int row, int d[3]) {
        if (oct) {
            const int ax = row / 10, p = row % 10, b = p >= 6 ? 3 : p >= 3 ? 2 : p >= 1 ? 1 : 0;
            d[0] = ax;
            d[1] = p - b * (b + 1) / 2;
            d[2] = b;
            return;
        }
        const int id = first + row, r = near ? 3 : 7, o = near ? 1 : 3;
        d[0] = id % r - o;
        d[1] = (id / r) % r - o;
        d[2] = id / (r * r) - o;
    };
    std::vector<int> todo;
    for (int row = 0; row < nd; ++row) {
        int d[3];
        offset_of(row, d);
        const bool is_near = std::abs(d[0]) <= 1 && std::abs(d[1]) <= 1 && std::abs(d[2]) <= 1;
        if (kind != kInterval || !is_near) todo.push_back(row);
    }
    unsigned nthr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned w = 0; w < nthr; ++w)
        th.emplace_back([&, w] {
            for (size_t t = w; t < todo.size(); t += nthr) {
                const int row = todo[t];
                int d[3];
                offset_of(row, d);
                kernel_spectrum(n_b, n, h, S, d, tab->data(), V, &all[size_t(row) * NWS]);
            }
        });
    for (auto& t : th) t.join();
    auto e = std::make_shared<SpecEntry>();
    e->device = device;
    const size_t elem = prec == LGF_FP64 ? sizeof(double) : sizeof(float);
    e->bytes = size_t(nd) * NWS * 2 * elem;
    (void)NW;
    cudaError_t ce = cudaMalloc(&e->ptr, e->bytes);
    if (ce != cudaSuccess) {
        e->ptr = nullptr;
        return fail(LGF_ERR_OOM, std::string("spectra allocation: ") + cudaGetErrorString(ce));
    }
    if (prec == LGF_FP64) {
        ce = cudaMemcpy(e->ptr, all.data(), e->bytes, cudaMemcpyHostToDevice);
    } else {
        std::vector<float> f(size_t(nd) * NWS * 2);
        for (size_t i = 0; i < all.size(); ++i) {
            f[2 * i] = float(all[i].real());
            f[2 * i + 1] = float(all[i].imag());
        }
        ce = cudaMemcpy(e->ptr, f.data(), e->bytes, cudaMemcpyHostToDevice);
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "spectra upload");
    e->has_tmap = !near && !oct && encode_table_map(*e, nd, NWS, prec);
    g_spec_cache[key] = e;
    out = e;
    return ok();
}

// ---------------------------------------------------------------------------
// Tree (Sec. 3.1): level-1 intervals are the blocks; the level-l index of a
// block b is floor(b / 2^(l-1)).  Sibling groups: index >> 1; a level's spectra
// are stored in slots group*8 + child, child = cx + 2 cy + 4 cz.

using I3 = std::array<int, 3>;

static inline int fdiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }
static inline I3 parent_of(const I3& a) { return {fdiv2(a[0]), fdiv2(a[1]), fdiv2(a[2])}; }
static inline int child_of(const I3& a) {
    return (a[0] - 2 * fdiv2(a[0])) + 2 * (a[1] - 2 * fdiv2(a[1])) + 4 * (a[2] - 2 * fdiv2(a[2]));
}
static inline uint64_t pack(const I3& a) {
    return (uint64_t(uint32_t(a[0] + (1 << 20))) << 42) | (uint64_t(uint32_t(a[1] + (1 << 20))) << 21) |
           uint64_t(uint32_t(a[2] + (1 << 20)));
}
static uint64_t morton(const I3& a, const I3& lo) {
    uint64_t m = 0;
    for (int bit = 0; bit < 21; ++bit)
        for (int ax = 0; ax < 3; ++ax)
            m |= uint64_t(((a[ax] - lo[ax]) >> bit) & 1) << (3 * bit + ax);
    return m;
}
static inline bool near(const I3& a, const I3& b) {
    return std::abs(a[0] - b[0]) <= 1 && std::abs(a[1] - b[1]) <= 1 && std::abs(a[2] - b[2]) <= 1;
}

struct Level {
    std::vector<I3> iv;                               // intervals (blocks at l = 0, 1)
    std::unordered_map<uint64_t, int> iv_index;
    std::vector<I3> groups;                           // Morton-sorted iv >> 1
    std::unordered_map<uint64_t, int> group_index;
    bool m2l = false;
    int slot(const I3& a) const { return group_index.at(pack(parent_of(a))) * 8 + child_of(a); }
};

struct DevLevel {
    int n_groups = 0;
    bool m2l = false;
    void* gs = nullptr;   // transform scratch of the run-time-size kernels
    void* fh = nullptr;
    void* uh = nullptr;
    void* ft = nullptr;
    void* ut = nullptr;
    int* gnbr = nullptr;
    int* order = nullptr;      // groups sorted by descending neighbour count
    R2CItem* r2c = nullptr;
    int n_r2c = 0;
    C2RItem* c2r = nullptr;
    int n_c2r = 0;
    // Reg and Interp items; the first n_reg_comp / n_int_comp belong to
    // problems whose passes sum with compensation, the rest sum plainly
    int* reg_child = nullptr;
    int* reg_parent = nullptr;
    int n_reg = 0, n_reg_comp = 0;
    int n_int_comp = 0;
    int* int_slot = nullptr;
    int* int_parent = nullptr;
    int* int_block = nullptr;       // level 1: the block of each item (output into the blocks)
    int n_int = 0;
    std::shared_ptr<SpecEntry> kh;
    bool oct = false;               // kh holds the 40 reflection representatives
    PersistPlan pp;                 // work lists and CTA ranges of the persistent products (FP32)
};

}  // namespace lgf

struct lgf_plan_s {
    int device = 0;
    int n_b = 0, n_I = 0, L = 0, n_max = 0, prec = LGF_FP32;
    int64_t n_blocks = 0, n_points = 0;
    int n_problems = 1;
    int S0 = 0, SI = 0, Lmac = 0;
    int near_kernel = 0, interval_kernel = 0;   // product-kernel variants (options)
    int single_stream = 0;
    int interp_mode = LGF_INTERP_NATIVE;   // Reg/Interp arithmetic (FP32 plans: tensor-core modes)
    // problems whose CUDA-core Reg/Interp passes sum with compensation (Dot2):
    // mode COMPENSATED, or NATIVE in an FP32 problem whose interaction lists
    // reach level 3 or higher (see build_plan)
    int comp_sums = 0;
    int* err = nullptr;                 // device flag: a bounded wait in a kernel ran out
    // SMs left to the levels >= 2 chain beside the persistent level-0 products
    // (-1: none; the chain then runs before and after them)
    int free_sms = 0;
    // level-0 transforms: 1 one CTA per block, 2 the persistent bulk-copy
    // form (FP32); grids of the persistent form and its block counters
    // ([0..1] forward, [2..3] inverse)
    int fft_kernel = 0;
    int symmetric_spectra = 0;          // option: 1 = reflection-reduced interval tables
    // block sizes without per-size kernels: the run-time-size kernels, their
    // twiddle tables (per transform length), the stencils in device memory
    // (per parent level) and the Reg / Interp scratch (n_ctas x 3 n_I^3 each)
    bool generic = false;
    std::map<int, void*> tw_dev;
    std::vector<void*> W_dev;
    void* gscratch[2] = {nullptr, nullptr};
    void* gslices = nullptr;   // Reg's per-child cubes (run-time-size kernels)
    int gctas = 0;
    int mac_gpc = 0;                    // option: sibling groups per CTA of the one-CTA-per-chunk products
    int cube_grid[2] = {0, 0};
    int* fft_ctr = nullptr;
    // the forward transform's input map, re-encoded when the input moves
    CUtensorMap in_map{};
    const void* in_map_src = nullptr;
    // levels 0 and 1 share the block grid and S0 = 2 n_b suffices for the
    // first n_b nodes of a level-1 interval: their products are summed into
    // one spectrum per block (one inverse FFT, no level-1 transforms)
    bool merged = true;
    std::vector<lgf::DevLevel> lev;
    std::vector<int64_t> pairs, intervals, groups;   // per level, for lgf_plan_get_stats
    void* W = nullptr;                  // device copy (unused by the kernels, kept for tools)
    // host copies of the 1D stencils passed by value to Reg / Interp, per
    // parent level l (the stencil between levels l and l - 1), and the
    // stencil size n_max of each
    std::vector<std::vector<float>> Wf;
    std::vector<std::vector<double>> Wd;
    std::vector<int> nmax_lv;
    int level_n_max(int l) const { return l < int(nmax_lv.size()) && nmax_lv[size_t(l)] > 0 ? nmax_lv[size_t(l)] : n_max; }
    lgf::C2RItem* out_items = nullptr;
    int n_out = 0;
    std::vector<void*> allocs;
    size_t bytes = 0;
    void* stage_f = nullptr;
    void* stage_u = nullptr;
    // lgf_solve_host_pipelined: a second staging pair, copy streams and the
    // events that order the two buffer pairs between copies and solves
    void* stage_f2 = nullptr;
    void* stage_u2 = nullptr;
    cudaStream_t copy_st[2] = {nullptr, nullptr};      // H2D, D2H
    cudaEvent_t pipe_ev[7] = {};                       // in_ready[2], solved[2], out_done[2], start
    // per-kernel event timing (lgf_plan_set_timing / lgf_plan_timings)
    std::vector<cudaEvent_t> ev;           // 2 * capacity events
    std::vector<const char*> ev_name;      // kernel name per recorded pair
    int ev_used = 0;
    int launches_last = 0;                 // kernels launched by the last solve
    // the level-1 chain and the level >= 2 chain run on their own streams,
    // forked from and joined into the caller's stream
    cudaStream_t aux[2] = {nullptr, nullptr};
    // join[0]: level-1 chain done; join[1]: levels >= 2 (or their upward part)
    // done; join[2]: level-0 products done; join[3]: level-0 inverse FFT done;
    // join[4]: levels >= 2 downward part done
    cudaEvent_t fork = nullptr, join[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // Workspace comes from the stream-ordered allocator on mem_st, so freeing
    // it waits for the plan's own last solve (done_ev, recorded at the end of
    // every solve on the caller's stream) instead of the whole device: a
    // server dropping an idle plan does not stall the requests in flight.
    cudaStream_t mem_st = nullptr;
    cudaEvent_t done_ev = nullptr;

    ~lgf_plan_s() {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        // a kernel-spectra table this plan alone still holds is freed with
        // cudaFree below (lev.clear()): let the plan's last solve finish first
        bool last_owner = false;
        for (const auto& D : lev) last_owner = last_owner || (D.kh && D.kh.use_count() == 1);
        if (last_owner && done_ev) cudaEventSynchronize(done_ev);
        if (mem_st) {
            if (done_ev) cudaStreamWaitEvent(mem_st, done_ev, 0);
            for (void* p : allocs) cudaFreeAsync(p, mem_st);
            for (void* p : {stage_f, stage_u, stage_f2, stage_u2})
                if (p) cudaFreeAsync(p, mem_st);
            cudaStreamDestroy(mem_st);   // returns at once; released when its work is done
        }
        if (done_ev) cudaEventDestroy(done_ev);
        for (cudaStream_t c : copy_st)
            if (c) cudaStreamDestroy(c);
        for (cudaEvent_t e : pipe_ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (cudaStream_t a : aux)
            if (a) cudaStreamDestroy(a);
        if (fork) cudaEventDestroy(fork);
        for (cudaEvent_t j : join)
            if (j) cudaEventDestroy(j);
        lev.clear();
        cudaSetDevice(cur);
    }
};

namespace lgf {

// Fault injection for tests: with LGF_FAULT_ALLOC_AT=k in the environment the
// k-th workspace allocation after the variable took that value (counting
// from 1) fails as if the device were out of memory.
static bool injected_alloc_failure() {
    static std::mutex mu;
    static std::string seen;
    static long long count = 0;
    const char* v = std::getenv("LGF_FAULT_ALLOC_AT");
    std::lock_guard<std::mutex> lock(mu);
    if (!v || !*v) {
        seen.clear();
        return false;
    }
    if (seen != v) {
        seen = v;
        count = 0;
    }
    return ++count == std::atoll(v);
}

static lgf_status dalloc(lgf_plan_s* P, size_t bytes, void** out, bool zero) {
    *out = nullptr;
    if (bytes == 0) return ok();
    if (injected_alloc_failure())
        return fail(LGF_ERR_OOM, "workspace allocation of " + std::to_string(bytes) + " bytes: injected failure");
    cudaError_t e = cudaMallocAsync(out, bytes, P->mem_st);
    if (e == cudaSuccess && zero) e = cudaMemsetAsync(*out, 0, bytes, P->mem_st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->mem_st);   // ready for use on any stream
    if (e != cudaSuccess) {
        if (*out) cudaFreeAsync(*out, P->mem_st);
        *out = nullptr;
        cudaGetLastError();
        return fail(LGF_ERR_OOM, "workspace allocation of " + std::to_string(bytes) + " bytes: " +
                                     cudaGetErrorString(e));
    }
    P->allocs.push_back(*out);
    P->bytes += bytes;
    return ok();
}

template <typename V>
static lgf_status upload(lgf_plan_s* P, const std::vector<V>& h, V** out) {
    *out = nullptr;
    if (h.empty()) return ok();
    void* p = nullptr;
    lgf_status s = dalloc(P, sizeof(V) * h.size(), &p, false);
    if (s != LGF_OK) return s;
    LGF_CUDA(cudaMemcpy(p, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice));
    *out = static_cast<V*>(p);
    return ok();
}

static std::mutex g_tw_mu;
static std::set<std::pair<int, int>> g_tw_done;

static lgf_status ensure_twiddles(int device, int prec) {
    std::lock_guard<std::mutex> lock(g_tw_mu);
    if (g_tw_done.count({device, prec})) return ok();
    // each unit holding transforms has its own copy of the tables
    cudaError_t e = prec == LGF_FP64 ? Launch<double>::init_twiddles() : Launch<float>::init_twiddles();
    if (e == cudaSuccess)
        e = prec == LGF_FP64 ? LaunchExt<double>::init_twiddles() : LaunchExt<float>::init_twiddles();
    if (e == cudaSuccess && prec == LGF_FP32) e = fft_large_init_twiddles();
    if (e != cudaSuccess) return cuda_fail(e, "twiddle upload");
    g_tw_done.insert({device, prec});
    return ok();
}

// One problem's tree, lists and item tables, with group, slot and block
// indices local to the problem.  A plan holds one or more problems: their
// tables are concatenated level by level with offsets, and since no list
// links two problems, each problem's result is the one it has alone.
struct HostLevel {
    int n_groups = 0;
    bool m2l = false;                          // interaction list not empty (level 0: near field, always)
    std::vector<int> gn;                       // n_groups x 27 neighbour groups, -1 = none
    std::vector<R2CItem> r2c;                  // src: block (l <= 1) or slot (l >= 2); dst: slot
    std::vector<int> iv_slot;                  // slot of each interval
    std::vector<int> reg_child, reg_parent;    // l >= 2: 8 children per parent (block at l = 2, else slot)
    std::vector<int> int_slot, int_parent;     // 1 <= l < Lmac
};

struct HostPlan {
    int L = 0, Lmac = 0;
    int64_t n_blocks = 0;
    std::vector<HostLevel> lev;                // levels 0..Lmac
    std::vector<int64_t> pairs, intervals, groups;   // levels 0..L
};

// Bounds checks of the tables a plan hands to its kernels, on the host before
// upload: every index a kernel dereferences lies inside the buffer it
// addresses.  A violation is an internal error and fails the plan.
static lgf_status check_range(const char* what, const std::vector<int>& v, long long lo, long long hi) {
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i] < lo || v[i] >= hi)
            return fail(LGF_ERR_INVALID_ARG, std::string("plan table check failed: ") + what + "[" + std::to_string(i) +
                                                 "] = " + std::to_string(v[i]) + " outside [" + std::to_string(lo) +
                                                 ", " + std::to_string(hi) + ")");
    return ok();
}

// Whether level l's products run in the persistent kernel: FP32 plans with
// interval_kernel 4 (or the default 0), at the interval levels and at level 0
// when it carries the merged level-0/level-1 products.  Its 24 warps share the
// groups of one frequency chunk, so by default a level needs at least 48
// groups (fewer leave warps idle; the one-CTA-per-chunk form is faster there).
static bool uses_persist(const lgf_plan_s* P, int l);
// The level-0 products leave free_sms SMs to a levels >= 2 chain beside them.
static bool shares_sms(const lgf_plan_s* P) {
    return P->free_sms > 0 && P->Lmac >= 2 && P->merged && uses_persist(P, 0);
}
static bool uses_persist(const lgf_plan_s* P, int l) {
    if (P->prec != LGF_FP32) return false;
    if (!persist_supported(l == 0 ? P->S0 : P->SI)) return false;
    if (P->interval_kernel != 0 && P->interval_kernel != 4 && P->interval_kernel != 5) return false;
    if (l == 0 && !P->merged) return false;
    // beside shared-SM level-0 products, levels >= 2 keep the
    // one-CTA-per-chunk form, which fits on the SMs left to them
    if (l >= 2 && shares_sms(P)) return false;
    return P->interval_kernel >= 4 || P->lev[size_t(l)].n_groups >= 48;
}

// Work lists of the persistent kernel for one level (see PersistPlan); the
// level's units (frequency chunk of 32, group position) are split at group
// boundaries into one range per CTA of about equal work (a unit weighs its
// pairs plus one for the group's set-up and stores).  The launch has one CTA
// per SM, less `free` SMs left to other kernels.
static lgf_status build_persist(lgf_plan_s* P, DevLevel& D, const std::vector<int>& gn, const std::vector<int>& ord,
                                int S, bool include_self, int free) {
    const int G = D.n_groups;
    std::vector<PairSrc> pairs;
    std::vector<int> start(size_t(G) + 1, 0);
    for (int pos = 0; pos < G; ++pos) {
        const int g = ord[size_t(pos)];
        for (int e = 0; e < 27; ++e) {
            const int q = gn[size_t(g) * 27 + e];
            if (q < 0 || (e == 13 && !include_self)) continue;
            const int ex = e % 3, ey = (e / 3) % 3, ez = e / 9;
            pairs.push_back({q, (2 * ex + 1) + 7 * (2 * ey + 1) + 49 * (2 * ez + 1)});
        }
        start[size_t(pos) + 1] = int(pairs.size());
    }
    {
        std::vector<int> src, centre;
        for (const PairSrc& q : pairs) {
            src.push_back(q.src);
            centre.push_back(q.centre);
        }
        lgf_status s;
        if ((s = check_range("pair source group", src, 0, G)) != LGF_OK) return s;
        // the 27 rows read around a centre stay inside the 343-row table
        if ((s = check_range("pair centre row", centre, 57, 343 - 57)) != LGF_OK) return s;
        for (int pos = 0; pos < G; ++pos)
            if (start[size_t(pos)] > start[size_t(pos) + 1]) return fail(LGF_ERR_INVALID_ARG, "plan table check failed: pair starts");
    }
    int n_sm = 0;
    LGF_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, P->device));
    const long long chunks = nws_of(S) / 32, n_cta = std::max(1, n_sm - std::max(0, free));
    std::vector<long long> pre(size_t(G) + 1, 0);
    for (int pos = 0; pos < G; ++pos)
        pre[size_t(pos) + 1] = pre[size_t(pos)] + (start[size_t(pos) + 1] - start[size_t(pos)]) + 1;
    // every CTA first takes q whole chunks (a chunk staged for only part of
    // its groups costs as much as a whole one), then about equal work of the
    // units of the chunks left over
    const long long Wg = pre[size_t(G)], q = chunks / n_cta, rc = q * n_cta, Wr = Wg * (chunks - rc);
    std::vector<long long> cut(size_t(n_cta) + 1);
    for (long long b = 0; b <= n_cta; ++b) {
        const long long T = (Wr * b) / n_cta;
        const long long c = std::min(T / Wg, chunks - rc);
        const long long pos = std::lower_bound(pre.begin(), pre.end(), T - c * Wg) - pre.begin();
        cut[size_t(b)] = std::min((rc + c) * G + std::min<long long>(pos, G), chunks * G);
    }
    cut[0] = rc * G;
    cut[size_t(n_cta)] = chunks * G;
    for (size_t b = 1; b < cut.size(); ++b) cut[b] = std::max(cut[b], cut[b - 1]);
    std::vector<long long> units(size_t(4 * n_cta));
    for (long long b = 0; b < n_cta; ++b) {
        units[size_t(4 * b)] = q * b;
        units[size_t(4 * b + 1)] = q * (b + 1);
        units[size_t(4 * b + 2)] = cut[size_t(b)];
        units[size_t(4 * b + 3)] = cut[size_t(b) + 1];
    }
    lgf_status s;
    PairSrc* dp = nullptr;
    int* ds = nullptr;
    long long* dc = nullptr;
    if ((s = upload(P, pairs, &dp)) != LGF_OK) return s;
    if ((s = upload(P, start, &ds)) != LGF_OK) return s;
    if ((s = upload(P, units, &dc)) != LGF_OK) return s;
    D.pp.pairs = dp;
    D.pp.start = ds;
    D.pp.order = D.order;
    D.pp.cta_units = dc;
    D.pp.n_groups = G;
    D.pp.n_cta = int(n_cta);
    D.pp.err = P->err;
    D.pp.packed = P->interval_kernel == 5 || P->interval_kernel == 0;
    return ok();
}

static lgf_status build_host(const int32_t* ijk, int64_t NB, int L, HostPlan& H) {
    H.L = L;
    H.n_blocks = NB;
    std::vector<I3> blocks(static_cast<size_t>(NB));
    std::unordered_map<uint64_t, int> bidx;
    for (int64_t b = 0; b < NB; ++b) {
        I3 v{ijk[3 * b], ijk[3 * b + 1], ijk[3 * b + 2]};
        for (int a = 0; a < 3; ++a)
            if (std::abs(v[a]) > (1 << 19)) return fail(LGF_ERR_INVALID_ARG, "block index out of range (|i| > 2^19)");
        if (!bidx.emplace(pack(v), int(b)).second)
            return fail(LGF_ERR_INVALID_ARG, "duplicate block in block_ijk at position " + std::to_string(b));
        blocks[size_t(b)] = v;
    }
    // levels 0..L: level 0 and 1 are the blocks
    std::vector<Level> lv(static_cast<size_t>(L) + 1);
    lv[0].iv = blocks;
    for (int l = 1; l <= L; ++l) {
        if (l == 1) {
            lv[1].iv = blocks;
        } else {
            std::unordered_set<uint64_t> seen;
            for (const I3& a : lv[size_t(l) - 1].iv) {
                I3 p = parent_of(a);
                if (seen.insert(pack(p)).second) lv[size_t(l)].iv.push_back(p);
            }
        }
        auto& L_ = lv[size_t(l)];
        for (size_t i = 0; i < L_.iv.size(); ++i) L_.iv_index[pack(L_.iv[i])] = int(i);
    }
    lv[0].iv_index = lv[1].iv_index;
    // the root level must have no interaction list
    {
        I3 lo = lv[size_t(L)].iv[0], hi = lo;
        for (const I3& a : lv[size_t(L)].iv)
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], a[k]);
                hi[k] = std::max(hi[k], a[k]);
            }
        if (hi[0] - lo[0] > 1 || hi[1] - lo[1] > 1 || hi[2] - lo[2] > 1) {
            int need = L;
            for (int l = L + 1; l < 40; ++l) {
                I3 a, b;
                for (int k = 0; k < 3; ++k) {
                    a[k] = lo[k];
                    b[k] = hi[k];
                    for (int s = L; s < l; ++s) {
                        a[k] = fdiv2(a[k]);
                        b[k] = fdiv2(b[k]);
                    }
                }
                if (b[0] - a[0] <= 1 && b[1] - a[1] <= 1 && b[2] - a[2] <= 1) {
                    need = l;
                    break;
                }
            }
            return fail(LGF_ERR_UNSUPPORTED,
                        "n_levels=" + std::to_string(L) + " leaves intervals at the root level that are not "
                        "mutually near (the root level would need its own interaction list); use n_levels >= " +
                            std::to_string(need));
        }
    }
    // interaction lists: sizes per level (level 0: near pairs); Lmac is the
    // highest level whose interaction list is not empty
    int Lmac = 0;
    H.pairs.assign(size_t(L) + 1, 0);
    H.intervals.assign(size_t(L) + 1, 0);
    H.groups.assign(size_t(L) + 1, 0);
    std::vector<bool> m2l(size_t(L) + 1, false);
    for (int l = 0; l <= L; ++l) H.intervals[size_t(l)] = int64_t(lv[size_t(l)].iv.size());
    for (const I3& a : lv[0].iv)
        for (int e = 0; e < 27; ++e) {
            const I3 q{a[0] + e % 3 - 1, a[1] + (e / 3) % 3 - 1, a[2] + e / 9 - 1};
            H.pairs[0] += lv[0].iv_index.count(pack(q));
        }
    for (int l = 1; l < L; ++l) {
        const auto& L_ = lv[size_t(l)];
        int64_t n = 0;
        for (const I3& a : L_.iv) {
            const I3 pp = parent_of(a);
            for (int e = 0; e < 216; ++e) {
                const int cx = e & 1, cy = (e >> 1) & 1, cz = (e >> 2) & 1, ee = e >> 3;
                const I3 q{2 * (pp[0] + ee % 3 - 1) + cx, 2 * (pp[1] + (ee / 3) % 3 - 1) + cy,
                           2 * (pp[2] + ee / 9 - 1) + cz};
                if (!near(a, q) && L_.iv_index.count(pack(q))) ++n;
            }
        }
        H.pairs[size_t(l)] = n;
        m2l[size_t(l)] = n > 0;
        if (n > 0) Lmac = l;
    }
    H.Lmac = Lmac;
    // sibling groups and slots for levels 0..Lmac
    for (int l = 0; l <= Lmac; ++l) {
        auto& L_ = lv[size_t(l)];
        std::unordered_set<uint64_t> seen;
        for (const I3& a : L_.iv) {
            I3 g = parent_of(a);
            if (seen.insert(pack(g)).second) L_.groups.push_back(g);
        }
        I3 lo = L_.groups[0];
        for (const I3& g : L_.groups)
            for (int k = 0; k < 3; ++k) lo[k] = std::min(lo[k], g[k]);
        std::sort(L_.groups.begin(), L_.groups.end(),
                  [&](const I3& a, const I3& b) { return morton(a, lo) < morton(b, lo); });
        for (size_t i = 0; i < L_.groups.size(); ++i) L_.group_index[pack(L_.groups[i])] = int(i);
        H.groups[size_t(l)] = int64_t(L_.groups.size());
    }
    // item tables
    H.lev.resize(size_t(Lmac) + 1);
    for (int l = 0; l <= Lmac; ++l) {
        const auto& L_ = lv[size_t(l)];
        HostLevel& T = H.lev[size_t(l)];
        T.n_groups = int(L_.groups.size());
        T.m2l = l == 0 || m2l[size_t(l)];
        T.gn.assign(size_t(T.n_groups) * 27, -1);
        for (int g = 0; g < T.n_groups; ++g)
            for (int e = 0; e < 27; ++e) {
                const I3& G = L_.groups[size_t(g)];
                I3 q{G[0] + e % 3 - 1, G[1] + (e / 3) % 3 - 1, G[2] + e / 9 - 1};
                auto it = L_.group_index.find(pack(q));
                if (it != L_.group_index.end()) T.gn[size_t(g) * 27 + e] = it->second;
            }
        for (size_t i = 0; i < L_.iv.size(); ++i) {
            const int slot = L_.slot(L_.iv[i]);
            T.iv_slot.push_back(slot);
            T.r2c.push_back({l <= 1 ? int(i) : slot, slot});
        }
        if (l >= 2) {
            const auto& Lc = lv[size_t(l) - 1];
            for (const I3& a : L_.iv) {
                T.reg_parent.push_back(L_.slot(a));
                const int cg = Lc.group_index.at(pack(a));
                for (int c = 0; c < 8; ++c) {
                    const I3 q{2 * a[0] + (c & 1), 2 * a[1] + ((c >> 1) & 1), 2 * a[2] + (c >> 2)};
                    auto it = Lc.iv_index.find(pack(q));
                    if (it == Lc.iv_index.end()) T.reg_child.push_back(-1);
                    else T.reg_child.push_back(l == 2 ? it->second : cg * 8 + c);
                }
            }
        }
        if (l >= 1 && l < Lmac) {
            const auto& Lp = lv[size_t(l) + 1];
            for (const I3& a : L_.iv) {
                T.int_slot.push_back(L_.slot(a));
                T.int_parent.push_back(Lp.slot(parent_of(a)));
            }
        }
    }
    return ok();
}

// Concatenates the problems' tables level by level and builds the device
// workspace.  A problem takes part in levels 0..its own Lmac; at a level where
// another problem has an interaction list but it has none, its products are
// exact zeros (all its pairs sit at near offsets, whose kernel is zero), so its
// result is unchanged.
static lgf_status build_plan(lgf_plan_s* P, const std::vector<HostPlan>& hp) {
    const int nb = P->n_b, nI = P->n_I;
    const size_t np = hp.size();
    int L = 0, Lmac = 0;
    for (const HostPlan& H : hp) {
        L = std::max(L, H.L);
        Lmac = std::max(Lmac, H.Lmac);
    }
    P->L = L;
    P->Lmac = Lmac;
    P->pairs.assign(size_t(L) + 1, 0);
    P->intervals.assign(size_t(L) + 1, 0);
    P->groups.assign(size_t(L) + 1, 0);
    for (const HostPlan& H : hp)
        for (int l = 0; l <= H.L; ++l) {
            P->pairs[size_t(l)] += H.pairs[size_t(l)];
            P->intervals[size_t(l)] += H.intervals[size_t(l)];
            P->groups[size_t(l)] += H.groups[size_t(l)];
        }
    // offsets: blocks per problem, groups per (level, problem); -1 = absent
    std::vector<int> boff(np, 0);
    for (size_t p = 1; p < np; ++p) boff[p] = boff[p - 1] + int(hp[p - 1].n_blocks);
    std::vector<std::vector<int>> goff(size_t(Lmac) + 1, std::vector<int>(np, -1));
    std::vector<int> ngroups(size_t(Lmac) + 1, 0);
    for (int l = 0; l <= Lmac; ++l)
        for (size_t p = 0; p < np; ++p)
            if (l <= hp[p].Lmac) {
                goff[size_t(l)][p] = ngroups[size_t(l)];
                ngroups[size_t(l)] += hp[p].lev[size_t(l)].n_groups;
            }
    const size_t elem = P->prec == LGF_FP64 ? sizeof(double) : sizeof(float);
    const size_t cplx = 2 * elem;
    const size_t n3 = size_t(nI) * nI * nI;
    {
        void* e = nullptr;
        lgf_status s = dalloc(P, sizeof(int), &e, true);
        if (s != LGF_OK) return s;
        P->err = static_cast<int*>(e);
    }
    // Compensated Reg/Interp sums (Dot2), decided per problem so that every
    // problem of a multi-problem plan gets the arithmetic it has alone: mode
    // COMPENSATED, or NATIVE in an FP32 problem whose interaction lists reach
    // level 3 or higher.  There a level-1 field is the sum of three or more
    // interpolated levels, and each Reg/Interp pass rounds FP32 sums of up to
    // n_max weights of mixed sign, the rounding amplified by the stencil's
    // Lebesgue constant (Sec. 2.5).  Measured on the 512^3 irregular 5-level
    // domain against the FP64 form: plain sums 1.04e-5, compensated 7.7e-6
    // (the 1e-5 FP32 tolerance), for 8% of the solve time; with products at
    // two levels only (the 128^3 torus) the transforms and products dominate
    // the error and the plain sums are kept, except for the block sizes of
    // the run-time-size kernels (n_b >= 18), whose interpolated fields are
    // summed from more terms: there the sums are compensated from the first
    // interpolated level on (measured, irregular three-level tori against
    // FP64: n_b = 18 plain 1.05e-5, compensated 7.9e-6; n_b = 20 1.17e-5 /
    // 9.7e-6; 2-6% of the solve time).
    std::vector<int> pcomp(np, 0);
    P->comp_sums = 0;
    for (size_t p = 0; p < np; ++p) {
        pcomp[p] = P->interp_mode == LGF_INTERP_COMPENSATED ||
                   (P->interp_mode == LGF_INTERP_NATIVE && P->prec == LGF_FP32 &&
                    (hp[p].Lmac >= 3 || (P->generic && hp[p].Lmac >= 2)));
        P->comp_sums += pcomp[p];
    }
    P->lev.resize(size_t(Lmac) + 1);
    for (int l = 0; l <= Lmac; ++l) {
        const auto& go = goff[size_t(l)];
        DevLevel& D = P->lev[size_t(l)];
        D.n_groups = ngroups[size_t(l)];
        bool any = false;
        for (size_t p = 0; p < np; ++p)
            if (go[p] >= 0) any = any || hp[p].lev[size_t(l)].m2l;
        D.m2l = (l == 0) || (any && !(l == 1 && P->merged));
        const size_t slots = size_t(D.n_groups) * 8;
        lgf_status s;
        if (D.m2l) {
            const int S = l == 0 ? P->S0 : P->SI;
            const size_t NWS = size_t(nws_of(S));
            if ((s = dalloc(P, slots * NWS * cplx, &D.fh, true)) != LGF_OK) return s;
            if ((s = dalloc(P, slots * NWS * cplx, &D.uh, false)) != LGF_OK) return s;
            std::vector<int> gn;
            std::vector<R2CItem> items;
            for (size_t p = 0; p < np; ++p) {
                if (go[p] < 0) continue;
                const HostLevel& T = hp[p].lev[size_t(l)];
                for (int v : T.gn) gn.push_back(v >= 0 ? v + go[p] : -1);
                for (const R2CItem& it : T.r2c)
                    items.push_back({l <= 1 ? it.src + boff[p] : it.src + 8 * go[p], it.dst + 8 * go[p]});
            }
            if ((s = check_range("neighbour group", gn, -1, D.n_groups)) != LGF_OK) return s;
            {
                std::vector<int> src, dst;
                for (const R2CItem& it : items) {
                    src.push_back(it.src);
                    dst.push_back(it.dst);
                }
                if ((s = check_range("forward FFT source", src, 0, l <= 1 ? P->n_blocks : static_cast<long long>(slots))) != LGF_OK)
                    return s;
                if ((s = check_range("forward FFT slot", dst, 0, static_cast<long long>(slots))) != LGF_OK) return s;
            }
            if ((s = upload(P, gn, &D.gnbr)) != LGF_OK) return s;
            {
                std::vector<int> cnt(size_t(D.n_groups), 0), ord(size_t(D.n_groups));
                for (int g = 0; g < D.n_groups; ++g) {
                    for (int e = 0; e < 27; ++e) cnt[size_t(g)] += gn[size_t(g) * 27 + e] >= 0;
                    ord[size_t(g)] = g;
                }
                std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cnt[size_t(a)] > cnt[size_t(b)]; });
                if ((s = upload(P, ord, &D.order)) != LGF_OK) return s;
                // with a levels >= 2 chain beside the level-0 products, level 0
                // leaves free_sms SMs to it
                int free = 0;
                if (l == 0 && Lmac >= 2) free = std::max(0, P->free_sms);
                if (uses_persist(P, l) && (s = build_persist(P, D, gn, ord, S, l == 0, free)) != LGF_OK) return s;
            }
            D.n_r2c = int(items.size());
            if ((s = upload(P, items, &D.r2c)) != LGF_OK) return s;
            const int h = l == 0 ? 1 : (1 << (l - 1));
            const int kind = l == 0 ? (P->merged ? kBlock : kNear) : kInterval;
            // reflection-reduced tables where the one-CTA-per-chunk products
            // run (the persistent kernel streams the half table by tensor copies)
            D.oct = P->symmetric_spectra == 1 && kind != kNear && !uses_persist(P, l) && !P->generic;
            if ((s = get_spectra(P->device, nb, S, h, kind, P->prec, D.kh, D.oct ? 1 : 0)) != LGF_OK) return s;
            D.pp.tmap = D.kh->has_tmap ? &D.kh->tmap : nullptr;
        }
        if (l >= 1 && !(l == 1 && P->merged && Lmac < 2)) {
            if ((s = dalloc(P, slots * n3 * elem, &D.ut, true)) != LGF_OK) return s;
            if (D.m2l) {
                std::vector<C2RItem> items;
                for (size_t p = 0; p < np; ++p) {
                    if (go[p] < 0) continue;
                    for (int slot : hp[p].lev[size_t(l)].iv_slot) items.push_back({slot + 8 * go[p], slot + 8 * go[p], -1});
                }
                D.n_c2r = int(items.size());
                for (const C2RItem& it : items)
                    if (it.src < 0 || it.src >= static_cast<long long>(slots) || it.dst < 0 || it.dst >= static_cast<long long>(slots))
                        return fail(LGF_ERR_INVALID_ARG, "plan table check failed: inverse FFT slot");
                if ((s = upload(P, items, &D.c2r)) != LGF_OK) return s;
            }
        }
        if (l >= 2) {
            if ((s = dalloc(P, slots * n3 * elem, &D.ft, true)) != LGF_OK) return s;
            std::vector<int> child, par;
            for (int pass : {1, 0}) {   // compensated problems' items first
                for (size_t p = 0; p < np; ++p) {
                    if (go[p] < 0 || pcomp[p] != pass) continue;
                    const HostLevel& T = hp[p].lev[size_t(l)];
                    for (int v : T.reg_parent) par.push_back(v + 8 * go[p]);
                    for (int c : T.reg_child)
                        child.push_back(c < 0 ? -1 : l == 2 ? c + boff[p] : c + 8 * goff[size_t(l) - 1][p]);
                }
                if (pass == 1) D.n_reg_comp = int(par.size());
            }
            D.n_reg = int(par.size());
            if ((s = check_range("Reg child", child, -1, l == 2 ? P->n_blocks : 8LL * ngroups[size_t(l) - 1])) != LGF_OK)
                return s;
            if ((s = check_range("Reg parent slot", par, 0, static_cast<long long>(slots))) != LGF_OK) return s;
            if ((s = upload(P, child, &D.reg_child)) != LGF_OK) return s;
            if ((s = upload(P, par, &D.reg_parent)) != LGF_OK) return s;
        }
        if (l >= 1 && l < Lmac) {
            std::vector<int> sl, pa, bl;
            for (int pass : {1, 0}) {   // compensated problems' items first
                for (size_t p = 0; p < np; ++p) {
                    if (go[p] < 0 || l >= hp[p].Lmac || pcomp[p] != pass) continue;
                    const HostLevel& T = hp[p].lev[size_t(l)];
                    for (int v : T.int_slot) sl.push_back(v + 8 * go[p]);
                    for (int v : T.int_parent) pa.push_back(v + 8 * goff[size_t(l) + 1][p]);
                    // level-1 intervals are the problem's blocks, in block order
                    if (l == 1)
                        for (size_t i = 0; i < T.int_slot.size(); ++i) bl.push_back(boff[p] + int(i));
                }
                if (pass == 1) D.n_int_comp = int(sl.size());
            }
            D.n_int = int(sl.size());
            if ((s = check_range("Interp slot", sl, 0, static_cast<long long>(slots))) != LGF_OK) return s;
            if ((s = check_range("Interp parent slot", pa, 0, 8LL * ngroups[size_t(l) + 1])) != LGF_OK) return s;
            if ((s = check_range("Interp block", bl, 0, P->n_blocks)) != LGF_OK) return s;
            if ((s = upload(P, sl, &D.int_slot)) != LGF_OK) return s;
            if ((s = upload(P, pa, &D.int_parent)) != LGF_OK) return s;
            if (l == 1 && (s = upload(P, bl, &D.int_block)) != LGF_OK) return s;
        }
    }
    // level-0 output items: block b from its level-0 slot, plus its level-1
    // field (same slot number within the problem, level-1 group offset)
    {
        std::vector<C2RItem> items;
        for (size_t p = 0; p < np; ++p) {
            const HostPlan& H = hp[p];
            const bool has_ut1 = P->merged ? H.Lmac >= 2 : H.Lmac >= 1;
            const std::vector<int>& s0 = H.lev[0].iv_slot;
            for (int64_t b = 0; b < H.n_blocks; ++b)
                items.push_back({s0[size_t(b)] + 8 * goff[0][p], int(b) + boff[p],
                                 has_ut1 ? s0[size_t(b)] + 8 * goff[1][p] : -1});
        }
        P->n_out = int(items.size());
        const long long s0 = 8LL * ngroups[0], s1 = Lmac >= 1 ? 8LL * ngroups[1] : 0;
        for (const C2RItem& it : items)
            if (it.src < 0 || it.src >= s0 || it.dst < 0 || it.dst >= P->n_blocks || it.aux >= s1 || it.aux < -1)
                return fail(LGF_ERR_INVALID_ARG, "plan table check failed: output item");
        lgf_status s = upload(P, items, &P->out_items);
        if (s != LGF_OK) return s;
    }
    // interpolation weights in the plan precision, per parent level
    {
        P->Wd.assign(size_t(L) + 1, {});
        P->Wf.assign(size_t(L) + 1, {});
        for (int l = 0; l <= L; ++l) {
            P->Wd[size_t(l)] = interp_weights(nb, P->level_n_max(l));
            P->Wf[size_t(l)].assign(P->Wd[size_t(l)].begin(), P->Wd[size_t(l)].end());
        }
        std::vector<double> W = interp_weights(nb, P->n_max);
        lgf_status s;
        if (P->prec == LGF_FP64) {
            double* d = nullptr;
            if ((s = upload(P, W, &d)) != LGF_OK) return s;
            P->W = d;
        } else {
            std::vector<float> wf(W.begin(), W.end());
            float* d = nullptr;
            if ((s = upload(P, wf, &d)) != LGF_OK) return s;
            P->W = d;
        }
    }
    if (P->generic) {
        lgf_status s;
        const bool f64 = P->prec == LGF_FP64;
        // twiddles (cos, sin)(2 pi m / S) of both transform lengths, FP64 values rounded once
        for (int S : {P->S0, P->SI}) {
            if (P->tw_dev.count(S)) continue;
            std::vector<double> t(2 * size_t(S));
            for (int m = 0; m < S; ++m) {
                const double a = 2.0 * M_PI * double(m) / double(S);
                t[2 * size_t(m)] = std::cos(a);
                t[2 * size_t(m) + 1] = std::sin(a);
            }
            void* d = nullptr;
            if (f64) {
                double* dd = nullptr;
                if ((s = upload(P, t, &dd)) != LGF_OK) return s;
                d = dd;
            } else {
                std::vector<float> tf(t.begin(), t.end());
                float* df = nullptr;
                if ((s = upload(P, tf, &df)) != LGF_OK) return s;
                d = df;
            }
            P->tw_dev[S] = d;
        }
        // the stencils of every parent level in device memory
        P->W_dev.assign(size_t(L) + 1, nullptr);
        for (int l = 2; l <= L; ++l) {
            if (f64) {
                double* d = nullptr;
                if ((s = upload(P, P->Wd[size_t(l)], &d)) != LGF_OK) return s;
                P->W_dev[size_t(l)] = d;
            } else {
                float* d = nullptr;
                if ((s = upload(P, P->Wf[size_t(l)], &d)) != LGF_OK) return s;
                P->W_dev[size_t(l)] = d;
            }
        }
        // transform scratch of each level: its larger item list, n_I planes
        // (none where the FP32 per-block transforms serve the level)
        for (int l = 0; l <= Lmac; ++l) {
            DevLevel& D = P->lev[size_t(l)];
            const int S = l == 0 ? P->S0 : P->SI;
            if (P->prec == LGF_FP32 && fft_large_supported(S, nb) && (l == 0 || fft_large_supported(S, nI)))
                continue;
            const size_t items = size_t(std::max({D.n_r2c, D.n_c2r, l == 0 ? P->n_out : 0}));
            if ((s = dalloc(P, items * size_t(nI) * size_t(S) * size_t(S / 2 + 1) * 2 * elem, &D.gs, false)) !=
                LGF_OK)
                return s;
        }
        // Reg / Interp scratch: two CTAs per SM, 2 cubes of n_I^3 each, and
        // Reg's slices for the largest level (8 per parent)
        if (Lmac >= 2) {
            int n_sm = 0;
            LGF_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, P->device));
            P->gctas = 2 * n_sm;
            const size_t bytes = size_t(P->gctas) * 2 * n3 * elem;
            for (void*& g : P->gscratch)
                if ((s = dalloc(P, bytes, &g, false)) != LGF_OK) return s;
            size_t parents = 0;
            for (int l = 2; l <= Lmac; ++l) parents = std::max(parents, size_t(P->lev[size_t(l)].n_reg));
            if ((s = dalloc(P, parents * 8 * n3 * elem, &P->gslices, false)) != LGF_OK) return s;
        }
    }
    return ok();
}

// A level's kernel table as a tensor map, when TMA loads are available for it
static const CUtensorMap* table_map(const DevLevel& D) { return D.kh && D.kh->has_tmap ? &D.kh->tmap : nullptr; }

// Runs one launch; with timing enabled, brackets it by an event pair on `st`.
template <typename F>
static cudaError_t timed(lgf_plan_s* P, const char* name, cudaStream_t st, F&& launch) {
    ++P->launches_last;
    const int k = P->ev_used;
    const bool rec = 2 * (k + 1) <= int(P->ev.size());
    if (rec) cudaEventRecord(P->ev[size_t(2 * k)], st);
    nvtxRangePushA(name);   // host-side range per launch, seen by profilers
    cudaError_t e = launch();
    nvtxRangePop();
    if (rec) {
        cudaEventRecord(P->ev[size_t(2 * k + 1)], st);
        P->ev_name[size_t(k)] = name;
        P->ev_used = k + 1;
    }
    return e;
}

template <typename T>
static lgf_status solve_impl(lgf_plan_s* P, const T* f, T* u, cudaStream_t st) {
    using Lc = Launch<T>;
    P->launches_last = 0;
    const int nb = P->n_b, nI = P->n_I;
    const int64_t n3 = int64_t(nI) * nI * nI, b3 = int64_t(nb) * nb * nb;
    auto& lev = P->lev;
    // the stencil between parent level l and level l - 1
    auto Wl = [&](int l) -> const T* {
        if constexpr (sizeof(T) == 8) return reinterpret_cast<const T*>(P->Wd[size_t(l)].data());
        else return reinterpret_cast<const T*>(P->Wf[size_t(l)].data());
    };
    // Transforms, products, Reg and Interp: the per-size kernels, or for the
    // block sizes without them the run-time-size kernels (generic.cu), which
    // pass the transforms through the level's other spectrum buffer.
    const bool gen = P->generic;
    using Gn = Generic<T>;
    // (the FP32 sizes 18 and 20 keep the per-block transforms, whose cubes fit)
    auto per_block = [&](int S, int n) { return sizeof(T) == 4 && fft_large_supported(S, n); };
    auto r2c_of = [&](int S, int n_in, const T* src, int64_t stride, DevLevel& D, cudaStream_t s) {
        if (gen && !per_block(S, n_in))
            return Gn::r2c(S, n_in, src, stride, D.r2c, D.n_r2c, D.fh, D.gs, P->tw_dev.at(S), s);
        return Lc::r2c(S, n_in, src, stride, D.r2c, D.n_r2c, D.fh, s);
    };
    auto c2r_of = [&](int S, int n_out, DevLevel& D, const C2RItem* items, int n, T* dst, int64_t ds, const T* add,
                      int add_n, int64_t as, cudaStream_t s) {
        if (gen && !per_block(S, n_out))
            return Gn::c2r(S, n_out, D.uh, items, n, D.gs, dst, ds, add, add_n, as, P->tw_dev.at(S), s);
        return Lc::c2r(S, n_out, D.uh, items, n, dst, ds, add, add_n, as, s);
    };
    auto reg_of = [&](int l, int nm, const T* src, int from_blocks, const int* child, const int* parent, int n, T* dst,
                      const T* W, int comp, cudaStream_t s) {
        if (gen)
            return Gn::reg(nb, src, from_blocks, child, parent, n, dst, static_cast<const T*>(P->W_dev[size_t(l)]),
                           comp, static_cast<T*>(P->gscratch[0]), static_cast<T*>(P->gslices), P->gctas, s);
        return Lc::reg(nb, nm, src, from_blocks, child, parent, n, dst, W, comp, s);
    };
    auto interp_of = [&](int lp, int nm, const int* slot, const int* parent, int n, T* out, const T* up, const T* W,
                         int accumulate, const int* block, int comp, cudaStream_t s) {
        if (gen)
            return Gn::interp(nb, slot, parent, n, out, up, static_cast<const T*>(P->W_dev[size_t(lp)]), accumulate,
                              block, comp, static_cast<T*>(P->gscratch[1]), P->gctas, s);
        return Lc::interp(nb, nm, slot, parent, n, out, up, W, accumulate, block, comp, s);
    };
    cudaError_t e;
    const int Lm = P->Lmac;
    const bool conc = !P->single_stream;
    cudaStream_t s1 = conc ? P->aux[0] : st, s2 = conc ? P->aux[1] : st;
    // The persistent level-0 kernel holds every SM until it ends, and anything
    // running beside it delays it.  With it, levels >= 2 are split: the upward
    // part (Reg, forward FFTs) runs beside the level-0 forward FFT, the
    // downward part (products, inverse FFTs, interpolation) beside the level-0
    // inverse FFT, and the level-2 field is finally interpolated straight into
    // the blocks.  Otherwise levels >= 2 run beside the level-0 products and
    // their level-1 field is added by the level-0 inverse FFT.
    const bool split = Lm >= 2 && uses_persist(P, 0) && P->free_sms < 0;
    auto record = [&](int k, cudaStream_t s) { return conc ? cudaEventRecord(P->join[k], s) : cudaSuccess; };
    auto wait = [&](cudaStream_t s, int k) { return conc ? cudaStreamWaitEvent(s, P->join[k], 0) : cudaSuccess; };
    // level-0 inverse FFT into u, plus the level-1 field add when given
    auto c2r0 = [&](const T* add) -> cudaError_t {
        if constexpr (std::is_same_v<T, float>)
            if (P->fft_kernel == 2)
                return c2r_cube(P->S0, nb, lev[0].uh, P->out_items, P->n_out, u, b3, add, nI, n3, P->cube_grid[1],
                                P->fft_ctr + 2, P->err, st);
        return c2r_of(P->S0, nb, lev[0], P->out_items, P->n_out, u, b3, add, nI, n3, st);
    };
    // fork: the other chains start after all prior work on the caller's stream
    if (conc && (Lm >= 2 || (Lm >= 1 && !P->merged))) {
        LGF_CUDA(cudaEventRecord(P->fork, st));
        if (!P->merged) LGF_CUDA(cudaStreamWaitEvent(s1, P->fork, 0));
        if (Lm >= 2) LGF_CUDA(cudaStreamWaitEvent(s2, P->fork, 0));
    }
    // Reg/Interp arithmetic: tensor-core modes, or the CUDA-core kernels with
    // plain or compensated sums
    const bool tc_mode = P->interp_mode != LGF_INTERP_NATIVE && P->interp_mode != LGF_INTERP_COMPENSATED &&
                         P->interp_mode != LGF_INTERP_PLAIN;
    // Interp of level l + 1 into the level-l items of D = lev[l] (see
    // Launch::interp) with the stencil of parent level l + 1; the CUDA-core
    // form in up to two launches: the items of problems with compensated
    // sums, then the others
    auto interp = [&](int l, T* out, const T* up, int accumulate, const int* block, cudaStream_t s) {
        DevLevel& D = lev[size_t(l)];
        const T* W = Wl(l + 1);
        const int nm = P->level_n_max(l + 1);
        if constexpr (sizeof(T) == 4) {
            if (tc_mode)
                return interp_tc(P->interp_mode, nb, D.int_slot, D.int_parent, D.n_int, out, up, W, accumulate, block,
                                 P->err, s);
        }
        cudaError_t r = cudaSuccess;
        const int nc = D.n_int_comp;
        if (nc > 0) r = interp_of(l + 1, nm, D.int_slot, D.int_parent, nc, out, up, W, accumulate, block, 1, s);
        if (nc > 0 && D.n_int > nc) ++P->launches_last;   // the second launch of this phase
        if (r == cudaSuccess && D.n_int > nc)
            r = interp_of(l + 1, nm, D.int_slot + nc, D.int_parent + nc, D.n_int - nc, out, up, W, accumulate,
                          block ? block + nc : nullptr, 0, s);
        return r;
    };
    // ---- levels >= 2 upward on s2: Reg from the level below, forward FFT
    auto up_part = [&]() -> lgf_status {
        for (int l = 2; l <= Lm; ++l) {
            DevLevel& D = lev[size_t(l)];
            const bool from_blocks = l == 2;
            e = timed(P, "reg", s2, [&] {
                const T* src = from_blocks ? f : static_cast<const T*>(lev[size_t(l) - 1].ft);
                const T* W = Wl(l);
                const int nm = P->level_n_max(l);
                if constexpr (sizeof(T) == 4) {
                    if (tc_mode)
                        return reg_tc(P->interp_mode, nb, src, from_blocks ? 1 : 0, D.reg_child, D.reg_parent, D.n_reg,
                                      static_cast<T*>(D.ft), W, P->err, s2);
                }
                cudaError_t r = cudaSuccess;
                const int nc = D.n_reg_comp;
                if (nc > 0)
                    r = reg_of(l, nm, src, from_blocks ? 1 : 0, D.reg_child, D.reg_parent, nc, static_cast<T*>(D.ft),
                               W, 1, s2);
                if (nc > 0 && D.n_reg > nc) ++P->launches_last;
                if (r == cudaSuccess && D.n_reg > nc)
                    r = reg_of(l, nm, src, from_blocks ? 1 : 0, D.reg_child + 8 * size_t(nc), D.reg_parent + nc,
                               D.n_reg - nc, static_cast<T*>(D.ft), W, 0, s2);
                return r;
            });
            if (e != cudaSuccess) return cuda_fail(e, "regularization");
            if (D.m2l) {
                e = timed(P, "r2c_interval", s2, [&] {
                    return r2c_of(P->SI, nI, static_cast<const T*>(D.ft), n3, D, s2);
                });
                if (e != cudaSuccess) return cuda_fail(e, "interval forward FFT");
            }
        }
        return ok();
    };
    // ---- levels >= 2 on s2: products, inverse FFTs and interpolation down to level 2
    auto down_part = [&]() -> lgf_status {
        for (int l = 2; l <= Lm; ++l) {
            DevLevel& D = lev[size_t(l)];
            if (!D.m2l) continue;
            e = timed(P, "mac_interval_l2plus", s2, [&] {
                if (uses_persist(P, l)) return Lc::mac_persist(D.fh, D.kh->ptr, D.uh, D.pp, P->SI, 0, s2);
                if (gen) return Gn::mac(D.fh, D.kh->ptr, D.uh, D.gnbr, D.n_groups, P->SI, 0, s2);
                return Lc::mac_interval(D.fh, D.kh->ptr, D.uh, D.gnbr, D.order, D.n_groups, P->SI, P->interval_kernel,
                                        0, table_map(D), P->err, s2, D.oct ? 1 : 0, P->mac_gpc);
            });
            if (e != cudaSuccess) return cuda_fail(e, "interaction-list products");
        }
        for (int l = Lm; l >= 2; --l) {
            DevLevel& D = lev[size_t(l)];
            if (D.m2l) {
                e = timed(P, "c2r_interval", s2, [&] {
                    return c2r_of(P->SI, nI, D, D.c2r, D.n_c2r, static_cast<T*>(D.ut), n3, nullptr, 0, 0, s2);
                });
                if (e != cudaSuccess) return cuda_fail(e, "interval inverse FFT");
            } else {
                e = cudaMemsetAsync(D.ut, 0, sizeof(T) * size_t(D.n_groups) * 8 * size_t(n3), s2);
                if (e != cudaSuccess) return cuda_fail(e, "clear level field");
            }
            if (l < Lm) {
                e = timed(P, "interp", s2, [&] {
                    return interp(l, static_cast<T*>(D.ut), static_cast<const T*>(lev[size_t(l) + 1].ut), 1, nullptr,
                                  s2);
                });
                if (e != cudaSuccess) return cuda_fail(e, "interpolation");
            }
        }
        return ok();
    };
    lgf_status r;
    if (split) {
        if ((r = up_part()) != LGF_OK) return r;
        LGF_CUDA(record(1, s2));
    }
    // ---- level 0 on the caller's stream: forward FFT, near-field products
    e = timed(P, "r2c_level0", st, [&] {
        if constexpr (std::is_same_v<T, float>)
            if (P->fft_kernel == 2) {
                if (P->in_map_src != f)
                    P->in_map_src = encode_rows_map(&P->in_map, f, P->n_blocks, nb) ? f : nullptr;
                if (P->in_map_src == f)
                    return r2c_cube(P->S0, nb, P->in_map, lev[0].r2c, lev[0].n_r2c, lev[0].fh, P->cube_grid[0],
                                    P->fft_ctr, P->err, st);
            }
        return r2c_of(P->S0, nb, f, b3, lev[0], st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "level-0 forward FFT");
    if (split) LGF_CUDA(wait(st, 1));
    if (P->merged) {
        e = timed(P, "mac_level01", st, [&] {
            // directly behind the forward FFT on st (no event between them):
            // launched early, it stages its first coefficient chunks meanwhile
            const int early = !split && P->ev.empty() ? 1 : 0;
            if (uses_persist(P, 0))
                return Lc::mac_persist(lev[0].fh, lev[0].kh->ptr, lev[0].uh, lev[0].pp, P->S0, early, st);
            if (gen) return Gn::mac(lev[0].fh, lev[0].kh->ptr, lev[0].uh, lev[0].gnbr, lev[0].n_groups, P->S0, 1, st);
            return Lc::mac_interval(lev[0].fh, lev[0].kh->ptr, lev[0].uh, lev[0].gnbr, lev[0].order, lev[0].n_groups,
                                    P->S0, P->interval_kernel == 3 ? 3 : 1, 1, table_map(lev[0]), P->err, st,
                                    lev[0].oct ? 1 : 0, P->mac_gpc);
        });
    } else {
        e = timed(P, "mac_level0", st, [&] {
            return Lc::mac_level0(lev[0].fh, lev[0].kh->ptr, lev[0].uh, lev[0].gnbr, lev[0].n_groups, P->S0,
                                  P->near_kernel, st);
        });
    }
    if (e != cudaSuccess) return cuda_fail(e, "near-field products");
    if (split) {
        // downward part after the level-0 products, beside the level-0 inverse FFT
        LGF_CUDA(record(2, st));
        LGF_CUDA(wait(s2, 2));
        if ((r = down_part()) != LGF_OK) return r;
        e = timed(P, "c2r_level0", st, [&] { return c2r0(nullptr); });
        if (e != cudaSuccess) return cuda_fail(e, "level-0 inverse FFT");
        LGF_CUDA(record(3, st));
        LGF_CUDA(wait(s2, 3));
        DevLevel& D = lev[1];
        e = timed(P, "interp", s2, [&] {
            return interp(1, u, static_cast<const T*>(lev[2].ut), 1, D.int_block, s2);
        });
        if (e != cudaSuccess) return cuda_fail(e, "interpolation");
        LGF_CUDA(record(4, s2));
        LGF_CUDA(wait(st, 4));
        return ok();
    }
    // ---- level 1 on s1: forward FFT, products, inverse FFT into u~1 (merged
    // form: already part of the level-0 products)
    if (Lm >= 1 && !P->merged) {
        DevLevel& D = lev[1];
        if (D.m2l) {
            e = timed(P, "r2c_interval", s1, [&] { return r2c_of(P->SI, nb, f, b3, D, s1); });
            if (e != cudaSuccess) return cuda_fail(e, "interval forward FFT");
            e = timed(P, "mac_interval_l1", s1, [&] {
                if (uses_persist(P, 1)) return Lc::mac_persist(D.fh, D.kh->ptr, D.uh, D.pp, P->SI, 0, s1);
                if (gen) return Gn::mac(D.fh, D.kh->ptr, D.uh, D.gnbr, D.n_groups, P->SI, 0, s1);
                return Lc::mac_interval(D.fh, D.kh->ptr, D.uh, D.gnbr, D.order, D.n_groups, P->SI, P->interval_kernel,
                                        0, table_map(D), P->err, s1, D.oct ? 1 : 0, P->mac_gpc);
            });
            if (e != cudaSuccess) return cuda_fail(e, "interaction-list products");
            e = timed(P, "c2r_interval", s1, [&] {
                return c2r_of(P->SI, nI, D, D.c2r, D.n_c2r, static_cast<T*>(D.ut), n3, nullptr, 0, 0, s1);
            });
            if (e != cudaSuccess) return cuda_fail(e, "interval inverse FFT");
        } else {
            e = cudaMemsetAsync(D.ut, 0, sizeof(T) * size_t(D.n_groups) * 8 * size_t(n3), s1);
            if (e != cudaSuccess) return cuda_fail(e, "clear level field");
        }
        LGF_CUDA(record(0, s1));
    }
    // ---- levels >= 2 on s2 beside the products; in the merged form u~1
    // holds only the interpolated level-2 field, stored at the chain's end
    if (Lm >= 2) {
        if ((r = up_part()) != LGF_OK) return r;
        if ((r = down_part()) != LGF_OK) return r;
        if (P->merged) {
            DevLevel& D = lev[1];
            e = timed(P, "interp", s2, [&] {
                return interp(1, static_cast<T*>(D.ut), static_cast<const T*>(lev[2].ut), 0, nullptr, s2);
            });
            if (e != cudaSuccess) return cuda_fail(e, "interpolation");
        }
        LGF_CUDA(record(1, s2));
    }
    // ---- join; in the separate form interpolate level 2 into the level-1
    // products' field (added to); then the level-0 output
    if (Lm >= 1 && !P->merged) LGF_CUDA(wait(st, 0));
    if (Lm >= 2) {
        LGF_CUDA(wait(st, 1));
        if (!P->merged) {
            DevLevel& D = lev[1];
            e = timed(P, "interp", st, [&] {
                return interp(1, static_cast<T*>(D.ut), static_cast<const T*>(lev[2].ut), 1, nullptr, st);
            });
            if (e != cudaSuccess) return cuda_fail(e, "interpolation");
        }
    }
    const bool has_ut1 = P->merged ? Lm >= 2 : Lm >= 1;
    const T* add = has_ut1 ? static_cast<const T*>(lev[1].ut) : nullptr;
    e = timed(P, "c2r_level0", st, [&] { return c2r0(add); });
    if (e != cudaSuccess) return cuda_fail(e, "level-0 inverse FFT");
    return ok();
}

static lgf_status check_device(const lgf_plan_s* P) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (cur != P->device)
        return fail(LGF_ERR_INVALID_ARG, "plan belongs to device " + std::to_string(P->device) +
                                             " but device " + std::to_string(cur) + " is current");
    return ok();
}

int plan_timing_capacity(const lgf_plan_s* plan) { return int(plan->ev.size() / 2); }

}  // namespace lgf

using namespace lgf;

extern "C" {

const char* lgf_last_error(void) { return g_err.c_str(); }

lgf_status lgf_interp_weights(int32_t n_b, int32_t n_max, double* W) {
    if (!W || n_b < 2 || n_max < 1 || n_max > n_b + 1)
        return fail(LGF_ERR_INVALID_ARG, "lgf_interp_weights: need W != NULL, n_b >= 2, 1 <= n_max <= n_b + 1");
    std::vector<double> v = interp_weights(n_b, n_max);
    std::memcpy(W, v.data(), sizeof(double) * v.size());
    return ok();
}

lgf_status lgf_plan_create(const int32_t* block_ijk, int64_t n_blocks, int32_t n_b, int32_t n_levels,
                           int32_t interp_order, int32_t precision, int32_t interp_mode, lgf_plan* out) {
    return lgf_plan_create_ex(block_ijk, n_blocks, n_b, n_levels, interp_order, precision, interp_mode,
                              nullptr, out);
}

static lgf_status create_plan(const int32_t* block_ijk, const int64_t* offsets, const int32_t* n_levels,
                              int32_t n_problems, int32_t n_b, int32_t interp_order, int32_t precision,
                              int32_t interp_mode, const lgf_plan_options* opts, lgf_plan* out) {
    if (!out) return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: out is NULL");
    *out = nullptr;
    if (!block_ijk || !offsets || !n_levels || n_problems < 1)
        return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: need block indices and at least one problem");
    if (offsets[0] != 0) return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create_multi: block_offsets[0] must be 0");
    for (int32_t p = 0; p < n_problems; ++p) {
        if (offsets[p + 1] - offsets[p] < 1)
            return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: need n_blocks >= 1 block indices (problem " +
                                                 std::to_string(p) + ")");
        if (n_levels[p] < 1 || n_levels[p] > 24)
            return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: need 1 <= n_levels <= 24");
    }
    const int64_t n_blocks = offsets[n_problems];
    if (n_blocks > (int64_t(1) << 26)) return fail(LGF_ERR_UNSUPPORTED, "lgf_plan_create: more than 2^26 blocks");
    if (n_b < 4 || n_b > 32 || n_b % 2 != 0)
        return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: n_b must be even, 4 <= n_b <= 32");
    if (interp_order < 0 || interp_order + 1 > n_b + 1)
        return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: need 0 <= interp_order and interp_order + 1 <= n_b + 1");
    if (precision != LGF_FP32 && precision != LGF_FP64)
        return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: precision must be LGF_FP32 or LGF_FP64");
    if (interp_mode < LGF_INTERP_NATIVE || interp_mode > LGF_INTERP_PLAIN)
        return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: interp_mode must be 0..5");
    if (interp_mode != LGF_INTERP_NATIVE && interp_mode != LGF_INTERP_PLAIN && precision != LGF_FP32)
        return fail(LGF_ERR_UNSUPPORTED, "lgf_plan_create: reduced-precision interpolation modes need an FP32 plan");
    if ((interp_mode == LGF_INTERP_BF16 || interp_mode == LGF_INTERP_FP16 || interp_mode == LGF_INTERP_BF16X3) &&
        n_b != 4 && n_b != 8 && n_b != 16)
        return fail(LGF_ERR_UNSUPPORTED, "lgf_plan_create: tensor-core interpolation modes need n_b 4, 8 or 16");
    auto P = std::make_unique<lgf_plan_s>();
    cudaError_t e = cudaGetDevice(&P->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    LGF_CUDA(cudaStreamCreateWithFlags(&P->mem_st, cudaStreamNonBlocking));
    LGF_CUDA(cudaEventCreateWithFlags(&P->done_ev, cudaEventDisableTiming));
    P->n_b = n_b;
    P->n_I = n_b + 1;
    P->n_max = interp_order + 1;
    P->prec = precision;
    P->interp_mode = interp_mode;
    P->n_blocks = n_blocks;
    P->n_problems = n_problems;
    P->n_points = n_blocks * int64_t(n_b) * n_b * n_b;
    P->S0 = s_level0(n_b);
    P->SI = s_interval(n_b);
    P->generic = !n_b_specialized(n_b);
    if (opts && opts->fft_size_interval != 0) {
        if (!s_interval_supported(n_b, opts->fft_size_interval))
            return fail(LGF_ERR_UNSUPPORTED, "lgf_plan_create: fft_size_interval " +
                                                 std::to_string(opts->fft_size_interval) +
                                                 " is not built for n_b = " + std::to_string(n_b));
        P->SI = opts->fft_size_interval;
    }
    if (opts) {
        if (opts->near_kernel != 0 || opts->interval_kernel < 0 || opts->interval_kernel > 5 ||
            opts->interval_kernel == 2)
            return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: near_kernel must be 0 and interval_kernel 0, 1, 3, 4 or 5");
        P->near_kernel = opts->near_kernel;
        P->interval_kernel = opts->interval_kernel;
        P->single_stream = opts->single_stream != 0;
        P->merged = opts->separate_level1 == 0;
        if (opts->free_sms < -1) return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: free_sms must be >= -1");
        P->free_sms = opts->free_sms;
        if (opts->fft_kernel < 0 || opts->fft_kernel > 2)
            return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: fft_kernel must be 0, 1 or 2");
        P->fft_kernel = opts->fft_kernel;
        if (opts->symmetric_spectra < 0 || opts->symmetric_spectra > 2)
            return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: symmetric_spectra must be 0, 1 or 2");
        P->symmetric_spectra = opts->symmetric_spectra;
        if (opts->mac_groups_per_cta < 0 || opts->mac_groups_per_cta > (1 << 20))
            return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: mac_groups_per_cta must be 0 .. 2^20");
        P->mac_gpc = opts->mac_groups_per_cta;
        // per-level interpolation orders: entry k is the stencil between
        // parent level k + 2 and level k + 1
        P->nmax_lv.assign(LGF_LEVEL_ORDERS + 2, 0);
        for (int k = 0; k < LGF_LEVEL_ORDERS; ++k) {
            const int o = opts->level_order[k];
            if (o == 0) continue;
            if (o < 0 || o + 1 > n_b + 1)
                return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: level_order[" + std::to_string(k) +
                                                     "] must be 0 or satisfy 1 <= order + 1 <= n_b + 1");
            P->nmax_lv[size_t(k) + 2] = o + 1;
        }
    }
    lgf_status s = ensure_twiddles(P->device, precision);
    if (s != LGF_OK) return s;
    std::vector<HostPlan> hp(static_cast<size_t>(n_problems));
    for (int32_t p = 0; p < n_problems; ++p) {
        s = build_host(block_ijk + 3 * offsets[p], offsets[p + 1] - offsets[p], n_levels[p], hp[size_t(p)]);
        if (s != LGF_OK) {
            if (n_problems > 1) fail(s, "problem " + std::to_string(p) + ": " + g_err);
            return s;
        }
    }
    if (P->free_sms == 0) {
        // Default schedule of the persistent products: when levels >= 2 carry
        // 7% or more of the level-0/1 pair work they get every SM after the
        // products (split); below that they run beside them on 24 SMs.
        // Measured on GB300 (ms, split / 24 SMs): 128^3 torus (ratio 0.05)
        // 0.280 / 0.252; 256^3 box (0.09) 2.254 / 2.307; 512^3 box (0.11)
        // 19.82 / 20.43; 512^3 irregular (0.12) 5.48 / 5.85.
        double main = 0, side = 0;
        for (const HostPlan& H : hp) {
            main += double(H.pairs[0] + (H.L >= 1 ? H.pairs[1] : 0)) * double(nw_of(P->S0));
            for (int l = 2; l <= H.L; ++l) side += double(H.pairs[size_t(l)]) * double(nw_of(P->SI));
        }
        P->free_sms = side > 0.07 * main ? -1 : 24;
    }
    s = build_plan(P.get(), hp);
    if (s != LGF_OK) return s;
    {
        const bool cube_ok = P->prec == LGF_FP32 && cube_fft_supported(P->S0, n_b);
        if (P->fft_kernel == 2 && !cube_ok)
            return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: fft_kernel 2 needs an FP32 plan with n_b 8 or 16");
        // default: the per-block form (measured on GB300, 128^3 torus: 28.4 /
        // 26.7 us forward / inverse in the step against 29.0 / 31.0 us)
        if (P->fft_kernel == 0) P->fft_kernel = 1;
        if (P->fft_kernel == 2) {
            int n_sm = 0;
            LGF_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, P->device));
            LGF_CUDA(cube_fft_grid(P->S0, n_b, false, n_sm, &P->cube_grid[0]));
            LGF_CUDA(cube_fft_grid(P->S0, n_b, true, n_sm, &P->cube_grid[1]));
            void* c = nullptr;
            if ((s = dalloc(P.get(), 4 * sizeof(int), &c, true)) != LGF_OK) return s;
            P->fft_ctr = static_cast<int*>(c);
        }
    }
    // In the split schedule the levels >= 2 chain (aux[1]) runs beside the
    // level-0 FFTs, which fill every SM: at the highest stream priority its
    // few CTAs go first (measured: 512^3 irregular 5.13e9 -> 5.25e9 points/s).
    // Beside the persistent products it keeps the default priority (there a
    // head start costs the level-0 forward FFT more than it gains).
    int prio_low = 0, prio_high = 0;
    LGF_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    LGF_CUDA(cudaStreamCreateWithFlags(&P->aux[0], cudaStreamNonBlocking));
    const bool split = P->free_sms < 0 && uses_persist(P.get(), 0);
    LGF_CUDA(cudaStreamCreateWithPriority(&P->aux[1], cudaStreamNonBlocking, split ? prio_high : prio_low));
    LGF_CUDA(cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming));
    for (auto& j : P->join) LGF_CUDA(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
    *out = P.release();
    return ok();
}

lgf_status lgf_plan_create_ex(const int32_t* block_ijk, int64_t n_blocks, int32_t n_b, int32_t n_levels,
                              int32_t interp_order, int32_t precision, int32_t interp_mode,
                              const lgf_plan_options* opts, lgf_plan* out) {
    if (!out) return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: out is NULL");
    *out = nullptr;
    if (!block_ijk || n_blocks < 1) return fail(LGF_ERR_INVALID_ARG, "lgf_plan_create: need n_blocks >= 1 block indices");
    const int64_t offsets[2] = {0, n_blocks};
    return create_plan(block_ijk, offsets, &n_levels, 1, n_b, interp_order, precision, interp_mode, opts, out);
}

lgf_status lgf_plan_create_multi(const int32_t* block_ijk, const int64_t* block_offsets, const int32_t* n_levels,
                                 int32_t n_problems, int32_t n_b, int32_t interp_order, int32_t precision,
                                 int32_t interp_mode, const lgf_plan_options* opts, lgf_plan* out) {
    return create_plan(block_ijk, block_offsets, n_levels, n_problems, n_b, interp_order, precision, interp_mode,
                       opts, out);
}

lgf_status lgf_plan_workspace_bytes(lgf_plan plan, size_t* bytes) {
    if (!plan || !bytes) return fail(LGF_ERR_INVALID_ARG, "lgf_plan_workspace_bytes: NULL argument");
    size_t b = plan->bytes;
    for (auto& D : plan->lev)
        if (D.kh) b += D.kh->bytes;
    *bytes = b;
    return ok();
}

lgf_status lgf_plan_get_stats(lgf_plan plan, lgf_plan_stats* st) {
    if (!plan || !st) return fail(LGF_ERR_INVALID_ARG, "lgf_plan_get_stats: NULL argument");
    std::memset(st, 0, sizeof(*st));
    st->n_points = plan->n_points;
    st->n_blocks = plan->n_blocks;
    st->n_levels = plan->L;
    st->top_product_level = plan->Lmac;
    st->fft_size_level0 = plan->S0;
    st->fft_size_interval = plan->SI;
    for (int l = 0; l <= plan->L && l <= LGF_MAX_LEVELS; ++l) {
        st->pairs[l] = plan->pairs[size_t(l)];
        st->intervals[l] = plan->intervals[size_t(l)];
        st->groups[l] = plan->groups[size_t(l)];
        if (l <= plan->Lmac && plan->lev[size_t(l)].m2l) st->nw[l] = nw_of(l == 0 ? plan->S0 : plan->SI);
    }
    st->merged_level01 = plan->merged ? 1 : 0;
    st->n_problems = plan->n_problems;
    st->persistent_ctas = uses_persist(plan, 0) ? plan->lev[0].pp.n_cta : 0;
    st->fft_kernel = plan->fft_kernel;
    st->compensated_interp = plan->comp_sums;
    if (plan->merged && plan->Lmac >= 1) st->nw[1] = nw_of(plan->S0);
    size_t b = 0;
    lgf_plan_workspace_bytes(plan, &b);
    st->workspace_bytes = int64_t(b);
    return ok();
}

lgf_status lgf_plan_points(lgf_plan plan, int64_t* n_points) {
    if (!plan || !n_points) return fail(LGF_ERR_INVALID_ARG, "lgf_plan_points: NULL argument");
    *n_points = plan->n_points;
    return ok();
}

lgf_status lgf_solve(lgf_plan plan, const void* f_dev, void* u_dev, void* stream) {
    if (!plan || !f_dev || !u_dev) return fail(LGF_ERR_INVALID_ARG, "lgf_solve: NULL argument");
    if (f_dev == u_dev) return fail(LGF_ERR_INVALID_ARG, "lgf_solve: f and u must not overlap");
    lgf_status s = check_device(plan);
    if (s != LGF_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    nvtxRangePushA("lgf_solve");
    const lgf_status r =
        plan->prec == LGF_FP64
            ? solve_impl<double>(plan, static_cast<const double*>(f_dev), static_cast<double*>(u_dev), st)
            : solve_impl<float>(plan, static_cast<const float*>(f_dev), static_cast<float*>(u_dev), st);
    nvtxRangePop();
    if (r == LGF_OK) {
        // the plan's completion marker (lgf_plan_sync, lgf_destroy); a solve
        // captured into a graph leaves it to the graph's owner
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        LGF_CUDA(cudaStreamIsCapturing(st, &cs));
        if (cs == cudaStreamCaptureStatusNone) LGF_CUDA(cudaEventRecord(plan->done_ev, st));
    }
    return r;
}

lgf_status lgf_solve_batch(const lgf_plan* plans, const void* const* f_dev, void* const* u_dev, int32_t n,
                           void* stream) {
    if (n < 0 || (n > 0 && (!plans || !f_dev || !u_dev)))
        return fail(LGF_ERR_INVALID_ARG, "lgf_solve_batch: bad arguments");
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < i; ++j)
            if (plans[i] == plans[j]) return fail(LGF_ERR_INVALID_ARG, "lgf_solve_batch: plans must be distinct");
    for (int32_t i = 0; i < n; ++i) {
        lgf_status s = lgf_solve(plans[i], f_dev[i], u_dev[i], stream);
        if (s != LGF_OK) return s;
    }
    return ok();
}

lgf_status lgf_solve_host(lgf_plan plan, const void* f_host, void* u_host, void* stream) {
    if (!plan || !f_host || !u_host) return fail(LGF_ERR_INVALID_ARG, "lgf_solve_host: NULL argument");
    lgf_status s = check_device(plan);
    if (s != LGF_OK) return s;
    const size_t bytes = size_t(plan->n_points) * (plan->prec == LGF_FP64 ? sizeof(double) : sizeof(float));
    if (!plan->stage_f) {
        cudaError_t e = cudaMallocAsync(&plan->stage_f, bytes, plan->mem_st);
        if (e == cudaSuccess) e = cudaMallocAsync(&plan->stage_u, bytes, plan->mem_st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(plan->mem_st);
        if (e != cudaSuccess) return fail(LGF_ERR_OOM, std::string("staging buffers: ") + cudaGetErrorString(e));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LGF_CUDA(cudaMemcpyAsync(plan->stage_f, f_host, bytes, cudaMemcpyHostToDevice, st));
    s = lgf_solve(plan, plan->stage_f, plan->stage_u, stream);
    if (s != LGF_OK) return s;
    LGF_CUDA(cudaMemcpyAsync(u_host, plan->stage_u, bytes, cudaMemcpyDeviceToHost, st));
    LGF_CUDA(cudaStreamSynchronize(st));
    return ok();
}

lgf_status lgf_solve_host_pipelined(lgf_plan plan, const void* const* f_host, void* const* u_host, int32_t n_steps,
                                    void* stream) {
    if (!plan || n_steps < 0 || (n_steps > 0 && (!f_host || !u_host)))
        return fail(LGF_ERR_INVALID_ARG, "lgf_solve_host_pipelined: bad arguments");
    for (int32_t k = 0; k < n_steps; ++k)
        if (!f_host[k] || !u_host[k]) return fail(LGF_ERR_INVALID_ARG, "lgf_solve_host_pipelined: NULL host buffer");
    lgf_status s = check_device(plan);
    if (s != LGF_OK) return s;
    if (n_steps == 0) return ok();
    const size_t bytes = size_t(plan->n_points) * (plan->prec == LGF_FP64 ? sizeof(double) : sizeof(float));
    if (!plan->stage_f2) {
        cudaError_t e = cudaSuccess;
        for (void** p : {&plan->stage_f, &plan->stage_u, &plan->stage_f2, &plan->stage_u2})
            if (!*p && e == cudaSuccess) e = cudaMallocAsync(p, bytes, plan->mem_st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(plan->mem_st);
        if (e != cudaSuccess) return fail(LGF_ERR_OOM, std::string("staging buffers: ") + cudaGetErrorString(e));
        for (cudaStream_t& c : plan->copy_st) LGF_CUDA(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
        for (cudaEvent_t& e2 : plan->pipe_ev) LGF_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStream_t h2d = plan->copy_st[0], d2h = plan->copy_st[1];
    cudaEvent_t* in_ready = plan->pipe_ev;
    cudaEvent_t* solved = plan->pipe_ev + 2;
    cudaEvent_t* out_done = plan->pipe_ev + 4;
    void* fd[2] = {plan->stage_f, plan->stage_f2};
    void* ud[2] = {plan->stage_u, plan->stage_u2};
    // the copies start after the work already queued on the caller's stream
    LGF_CUDA(cudaEventRecord(plan->pipe_ev[6], st));
    LGF_CUDA(cudaStreamWaitEvent(h2d, plan->pipe_ev[6], 0));
    for (int32_t k = 0; k < n_steps; ++k) {
        const int b = k & 1;
        // input k into buffer b once the solve of step k - 2 has read it
        if (k >= 2) LGF_CUDA(cudaStreamWaitEvent(h2d, solved[b], 0));
        LGF_CUDA(cudaMemcpyAsync(fd[b], f_host[k], bytes, cudaMemcpyHostToDevice, h2d));
        LGF_CUDA(cudaEventRecord(in_ready[b], h2d));
        // solve k once its input is in and step k - 2's result has left ud[b]
        LGF_CUDA(cudaStreamWaitEvent(st, in_ready[b], 0));
        if (k >= 2) LGF_CUDA(cudaStreamWaitEvent(st, out_done[b], 0));
        s = lgf_solve(plan, fd[b], ud[b], stream);
        if (s != LGF_OK) return s;
        LGF_CUDA(cudaEventRecord(solved[b], st));
        // result k out behind its solve
        LGF_CUDA(cudaStreamWaitEvent(d2h, solved[b], 0));
        LGF_CUDA(cudaMemcpyAsync(u_host[k], ud[b], bytes, cudaMemcpyDeviceToHost, d2h));
        LGF_CUDA(cudaEventRecord(out_done[b], d2h));
    }
    LGF_CUDA(cudaStreamSynchronize(d2h));
    LGF_CUDA(cudaStreamSynchronize(st));
    return ok();
}

lgf_status lgf_plan_set_timing(lgf_plan plan, int32_t capacity) {
    if (!plan || capacity < 0 || capacity > (1 << 16))
        return fail(LGF_ERR_INVALID_ARG, "lgf_plan_set_timing: need a plan and 0 <= capacity <= 65536");
    lgf_status s = check_device(plan);
    if (s != LGF_OK) return s;
    LGF_CUDA(cudaDeviceSynchronize());
    for (cudaEvent_t e : plan->ev) cudaEventDestroy(e);
    plan->ev.clear();
    plan->ev_name.assign(size_t(capacity), nullptr);
    plan->ev_used = 0;
    for (int i = 0; i < 2 * capacity; ++i) {
        cudaEvent_t e;
        LGF_CUDA(cudaEventCreate(&e));
        plan->ev.push_back(e);
    }
    return ok();
}

lgf_status lgf_plan_timings(lgf_plan plan, int32_t max_kernels, int32_t* n_kernels, char* names,
                            double* total_ms, int32_t* count, int32_t* launches_per_solve) {
    if (!plan || !n_kernels || max_kernels < 0 || (max_kernels > 0 && (!names || !total_ms || !count)))
        return fail(LGF_ERR_INVALID_ARG, "lgf_plan_timings: bad arguments");
    lgf_status s = check_device(plan);
    if (s != LGF_OK) return s;
    std::vector<std::string> nm;
    std::vector<double> tot;
    std::vector<int> cnt;
    for (int k = 0; k < plan->ev_used; ++k) {
        LGF_CUDA(cudaEventSynchronize(plan->ev[size_t(2 * k + 1)]));
        float ms = 0.f;
        LGF_CUDA(cudaEventElapsedTime(&ms, plan->ev[size_t(2 * k)], plan->ev[size_t(2 * k + 1)]));
        const std::string name = plan->ev_name[size_t(k)];
        size_t j = 0;
        while (j < nm.size() && nm[j] != name) ++j;
        if (j == nm.size()) {
            nm.push_back(name);
            tot.push_back(0.0);
            cnt.push_back(0);
        }
        tot[j] += ms;
        cnt[j] += 1;
    }
    *n_kernels = int32_t(nm.size());
    for (size_t j = 0; j < nm.size() && int32_t(j) < max_kernels; ++j) {
        std::memset(names + 32 * j, 0, 32);
        std::strncpy(names + 32 * j, nm[j].c_str(), 31);
        total_ms[j] = tot[j];
        count[j] = cnt[j];
    }
    if (launches_per_solve) *launches_per_solve = plan->launches_last;
    plan->ev_used = 0;
    return ok();
}

lgf_status lgf_plan_sync(lgf_plan plan) {
    if (!plan) return fail(LGF_ERR_INVALID_ARG, "lgf_plan_sync: NULL plan");
    lgf_status s = check_device(plan);
    if (s != LGF_OK) return s;
    LGF_CUDA(cudaEventSynchronize(plan->done_ev));
    if (plan->err) {
        int flag = 0;
        LGF_CUDA(cudaMemcpy(&flag, plan->err, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            LGF_CUDA(cudaMemset(plan->err, 0, sizeof(int)));
            return fail(LGF_ERR_CUDA, "lgf_plan_sync: a wait inside a product kernel ran out (results invalid)");
        }
    }
    return ok();
}

lgf_status lgf_destroy(lgf_plan plan) {
    if (!plan) return fail(LGF_ERR_INVALID_ARG, "lgf_destroy: NULL plan");
    delete plan;
    return ok();
}

}  // extern "C"
