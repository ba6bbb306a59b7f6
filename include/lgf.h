/*
 * lgf.h - C ABI of the GB300 LGF fast multipole solver.
 *
 * Solves the discrete Poisson problem  L u = f  on an unbounded 3D lattice
 * (Eq. dpoisson: L is the 7-point Laplacian with unit spacing), where f is
 * supported on a set of equal cubic blocks of n_b^3 points (Sec. 2.3), and u
 * is wanted on the same blocks.  The solution is the lattice convolution
 * u = G * f with the lattice Green's function G (Eq. dpoissonsoln), evaluated
 * by the Fast Lattice Green's Function method of Sec. 3.1: block and interval
 * convolutions done as zero-padded FFT convolutions against precomputed
 * kernel spectra (Sec. 2.2, Eq. precomp), a multilevel octree of interpolation
 * intervals with n_I = n_b + 1 equispaced nodes per axis (Sec. 4), Lagrange
 * interpolation with at most n_max = interp_order + 1 nodes per point (Sec. 2.5)
 * and its adjoint for regularization (Sec. 2.4).
 *
 * Data layout (caller side).  A field is n_blocks * n_b^3 values of the plan's
 * precision (float for LGF_FP32, double for LGF_FP64).  Block b (in the order
 * of block_ijk given at plan creation) owns values [b*n_b^3, (b+1)*n_b^3); its
 * point (i, j, k) is value i + n_b*(j + n_b*k) and sits at lattice point
 * block_ijk[b]*n_b + (i, j, k).
 *
 * Errors.  Every call returns an lgf_status; nothing else crosses the ABI.
 * lgf_last_error() returns a message for the calling thread's last failure.
 * Launch errors surface at the call; faults inside an asynchronous solve
 * surface at lgf_plan_sync() or at the next CUDA call on that stream.
 *
 * Concurrency.  A plan owns its device workspace, so one plan must not run two
 * solves at once (two streams, or two host threads).  Different plans are
 * independent.  Kernel spectra are shared between plans with equal (n_b,
 * precision) through a reference-counted cache; its entries live until the
 * last plan using them is destroyed.
 *
 * Device.  A plan is bound to the CUDA device current at lgf_plan_create; all
 * later calls on it must run with that device current.
 */
#ifndef LGF_H
#define LGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lgf_plan_s *lgf_plan;

typedef enum {
    LGF_OK = 0,
    LGF_ERR_INVALID_ARG = 1,   /* bad pointer, size, duplicate block, ...     */
    LGF_ERR_UNSUPPORTED = 2,   /* valid request the library does not handle    */
    LGF_ERR_OOM = 3,           /* device or host allocation failed            */
    LGF_ERR_CUDA = 4,          /* CUDA runtime error (message has details)     */
    LGF_ERR_TIMEOUT = 5,       /* a bounded device wait ran out               */
    LGF_ERR_BUDGET = 6         /* request exceeds a caller-given memory budget */
} lgf_status;

typedef enum { LGF_FP64 = 0, LGF_FP32 = 1 } lgf_precision;

/* Arithmetic of the regularization / interpolation contractions (Eqs. alg_reg,
 * alg_interp).  NATIVE uses the plan precision on the CUDA cores; in an FP32
 * plan whose interaction lists reach level 3 or higher (four or more levels)
 * it sums with compensation, as COMPENSATED below, because there a level-1
 * field carries three or more interpolated levels whose FP32 roundings,
 * amplified by the stencil's Lebesgue constant (Sec. 2.5), approach the 1e-5
 * relative tolerance (5-level 512^3 domain: 1.04e-5 plain, 7.7e-6
 * compensated, measured against the FP64 form); for n_b >= 18 it does so
 * from level 2 on (three-level irregular tori, n_b = 18: 1.05e-5 plain,
 * 7.9e-6 compensated).  PLAIN forces plain sums in
 * the plan precision at any depth.  The others
 * (FP32 plans only) run each axis pass as a tensor-core GEMM (tcgen05.mma)
 * with FP32 accumulation; the field between passes stays FP32 and only the
 * MMA inputs (field values and weights) are rounded:
 *   LGF_INTERP_BF16    BF16 inputs (8-bit significand)
 *   LGF_INTERP_FP16    FP16 inputs (11-bit significand; magnitudes above
 *                      65504 overflow: fields of order 1e4 or more need NATIVE)
 *   LGF_INTERP_BF16X3  inputs split into three BF16 parts, six partial
 *                      products: close to FP32 accuracy
 * Relative errors against the FP64 form, measured: in trees of up to 4
 * levels BF16 0.09-0.12 and FP16 1.1e-2-1.3e-2, inside 48 u (u = 2^-8 BF16,
 * 2^-11 FP16: up to 12 rounded passes, each amplified by the order-8
 * stencil's Lebesgue constant of about 3); that bound holds to 4 levels only:
 * on the 5-level 512^3 domain BF16 gives 0.40 and FP16 5.6e-2, as each
 * further level adds six rounded passes amplified through the levels below.
 * No reduced-precision mode meets the 1e-5 FP32 tolerance at 5 levels.
 * and, on the CUDA cores:
 *   LGF_INTERP_COMPENSATED  FP32 passes whose dot products carry the exact
 *                      rounding error of every product and sum (FMA-based
 *                      TwoProduct and TwoSum, accumulated as in Ogita, Rump
 *                      and Oishi's Dot2): each pass's output is its sum in
 *                      twice the working precision, rounded once.  Several
 *                      times the arithmetic of NATIVE in these small kernels;
 *                      for deep FP32 trees where the interpolation passes'
 *                      roundings, amplified by the stencil, approach the
 *                      tolerance */
typedef enum {
    LGF_INTERP_NATIVE = 0,
    LGF_INTERP_BF16 = 1,
    LGF_INTERP_FP16 = 2,
    LGF_INTERP_BF16X3 = 3,
    LGF_INTERP_COMPENSATED = 4,
    LGF_INTERP_PLAIN = 5
} lgf_interp_mode;

/*
 * lgf_plan_create - build the tree, lists, interpolation stencils and kernel
 * spectra for one block set (Sec. 3.1 Step 0 and Sec. 3.1 lists), and
 * allocate the device workspace of a solve.
 *
 *   block_ijk     host array, n_blocks x 3 int32 block indices (x, y, z);
 *                 unique; copied, the caller keeps ownership
 *   n_blocks      >= 1
 *   n_b           points per block edge, even, 4 <= n_b <= 32 (odd or out of
 *                 range: LGF_ERR_INVALID_ARG).  4 .. 16 run kernels built per
 *                 size (transforms in shared memory; in FP32 also 18 and 20);
 *                 the other steps of 18 .. 32 run kernels with run-time sizes
 *                 (transforms one axis per launch through a device scratch),
 *                 2-4 times slower per point.  The
 *                 tensor-core interpolation modes need 4, 8 or 16.
 *   n_levels      L >= 1: the leaves are level 1 and the root level is L
 *                 (Sec. 3.1).  Level L must hold intervals that are all near
 *                 one another (at most two per axis, aligned); otherwise
 *                 LGF_ERR_UNSUPPORTED with a message naming the needed depth.
 *   interp_order  polynomial degree p of the interpolation; n_max = p + 1
 *                 nodes are used per point, 1 <= n_max <= n_b + 1
 *   precision     LGF_FP32 or LGF_FP64 (FFTs, products and interpolation);
 *                 the LGF values and spectra are always generated in FP64
 *   interp_mode   LGF_INTERP_NATIVE or LGF_INTERP_PLAIN, or for FP32 plans
 *                 LGF_INTERP_BF16, LGF_INTERP_FP16, LGF_INTERP_BF16X3,
 *                 LGF_INTERP_COMPENSATED
 *                 (LGF_ERR_UNSUPPORTED for FP64 plans)
 *   out           receives the plan
 *
 * Runs on the host plus uploads on the current device; synchronous.
 */
lgf_status lgf_plan_create(const int32_t *block_ijk, int64_t n_blocks, int32_t n_b,
                           int32_t n_levels, int32_t interp_order, int32_t precision,
                           int32_t interp_mode, lgf_plan *out);

/*
 * Tuning options (zero-initialise for the defaults).
 *   fft_size_interval  FFT length per axis S_I at levels >= 1 (Sec. 2.2: any
 *                      S_I >= 2 n_I - 1 gives the same linear convolution).
 *                      0 = default.  Supported: n_b = 4: 10; 6: 16; 8: 17,
 *                      18; 10: 24; 12: 28; 14: 32; 16: 33, 34, 36; 18: 40;
 *                      20 .. 32: 2 n_b + 2 (the default).  The level-0 length
 *                      is 2 n_b.
 *   near_kernel        must be 0 (one product kernel for the level-0 near
 *                      field of the separate form: the 4^3 source blocks of a
 *                      sibling group, fully unrolled)
 *   interval_kernel    product kernel of levels >= 1 (and of the merged
 *                      level-0/1 pass): 0 = default (5 for FP32 plans where a
 *                      level has >= 48 sibling groups; elsewhere one CTA per
 *                      (frequency chunk, group range) with the packed FP32
 *                      products of form 5, 8 warps), 1 = one frequency per
 *                      thread, one CTA per (frequency chunk, group range), one
 *                      FMA per real product, 3 = two sibling groups per warp
 *                      sharing coefficient loads (2 is not a form: the two-
 *                      frequencies-per-thread form lost everywhere and was
 *                      removed), 4 = persistent: one CTA per SM,
 *                      each taking whole frequency chunks and then an equal
 *                      share of the chunks left over, coefficient chunks
 *                      staged by tensor copies into two shared-memory buffers,
 *                      5 = form 4 with the products as packed two-wide FP32
 *                      FMAs (fma.rn.f32x2), 16 warps per CTA
 *                      (3, 4 and 5: FP32 only; FP64 plans use 1).  A wait
 *                      in forms 4 and 5 that runs out (about 2 s) sets a flag
 *                      that lgf_plan_sync reports as LGF_ERR_CUDA.
 *   single_stream      1 = run every kernel of a solve on the caller's stream;
 *                      0 (default) = the level-1 chain and the levels >= 2
 *                      chain run on two plan-owned streams forked from and
 *                      joined into the caller's stream
 *   separate_level1    0 (default): the level-1 interaction list is summed
 *                      into the level-0 spectra.  Level-1 nodes are the grid
 *                      points and only the first n_b nodes of a level-1
 *                      interval are used (Sec. 4), so the level-0 transform
 *                      length 2 n_b already gives the exact level-1
 *                      convolution; by linearity both levels then share one
 *                      forward FFT, one product pass over the 6^3 blocks of
 *                      the parent neighbourhood (343 kernel offsets) and one
 *                      inverse FFT.  1: separate level-1 transforms of length
 *                      S_I, as the level interactions of Sec. 3.1 are listed.
 *   free_sms           schedule of the persistent products (interval_kernel
 *                      form 4): -1 = they take every SM and levels >= 2 run
 *                      before and after them; k > 0 = they take all but k SMs
 *                      and levels >= 2 run beside them on the rest; 0 = the
 *                      library's choice
 *   fft_kernel         level-0 forward and inverse FFTs: 1 = one CTA per block
 *                      (the input and output cubes through per-thread loads
 *                      and stores); 2 = persistent, one CTA per SM taking
 *                      blocks from a counter, the whole padded cube in shared
 *                      memory, each block's input, spectrum and output moved
 *                      by bulk copies that overlap the neighbouring blocks'
 *                      passes, each line transform split into output classes
 *                      (FP32 plans with n_b 8 or 16); 0 = 1 (the faster form
 *                      as measured)
 *   level_order        per-level interpolation orders (Sec. 4 notes that the
 *                      interval sizes and stencils may be tuned per level):
 *                      level_order[k] is the polynomial degree of the stencil
 *                      between parent level k + 2 and level k + 1 (Interp
 *                      from level k + 2, and Reg into it), 1 <= order + 1 <=
 *                      n_b + 1; 0 = interp_order.  Levels above
 *                      LGF_LEVEL_ORDERS + 1 use interp_order.
 *   symmetric_spectra  1: the levels whose products run one CTA per
 *                      frequency chunk (not the persistent form) store only
 *                      the 40 representatives of the 343 kernel offsets under
 *                      the reflections and axis exchanges that leave G
 *                      unchanged (Sec. 3.2: a reflected offset's spectrum is
 *                      the representative's at reflected frequencies; the
 *                      kernel vector is centred on index 0, so no twiddle is
 *                      needed), 4.3x fewer rows than the 172-row half table;
 *                      the products gather each offset's coefficients from
 *                      its representative.  0 / 2: the half tables.
 *   mac_groups_per_cta the interaction-list chunk of the one-CTA-per-chunk
 *                      products: sibling groups (each with its list of
 *                      neighbour groups) a CTA takes for one frequency chunk,
 *                      rounded up to whole warps; 0 = chosen from the level's
 *                      size (about four waves of CTAs)
 * All variants compute the same sums (Eq. alg_mult); they differ only in
 * scheduling.
 */
#define LGF_LEVEL_ORDERS 8
typedef struct {
    int32_t fft_size_interval;
    int32_t near_kernel;
    int32_t interval_kernel;
    int32_t single_stream;
    int32_t separate_level1;
    int32_t free_sms;
    int32_t fft_kernel;
    int32_t level_order[LGF_LEVEL_ORDERS];
    int32_t symmetric_spectra;
    int32_t mac_groups_per_cta;
    int32_t reserved[7];
} lgf_plan_options;

/* lgf_plan_create with options (NULL = defaults). */
lgf_status lgf_plan_create_ex(const int32_t *block_ijk, int64_t n_blocks, int32_t n_b,
                              int32_t n_levels, int32_t interp_order, int32_t precision,
                              int32_t interp_mode, const lgf_plan_options *opts, lgf_plan *out);

/*
 * lgf_plan_create_multi - one plan over n_problems independent problems that
 * share n_b, the interpolation order and the precision (batched solves of
 * uneven domains).  Problem p owns blocks block_offsets[p] ..
 * block_offsets[p+1]-1 of block_ijk (its own index space: problems may reuse
 * block indices) and has its own level count n_levels[p].  No list links two
 * problems, so each problem's u is the one a plan of it alone computes (Sec.
 * 3.1 applied per problem); the tables of all problems are concatenated, so
 * one lgf_solve runs one launch per phase for the whole set.
 *   block_offsets  n_problems + 1 ascending offsets, block_offsets[0] = 0,
 *                  at least one block per problem
 *   n_levels       n_problems level counts (each as in lgf_plan_create)
 *   f and u of lgf_solve: the problems' blocks back to back in this order.
 * Errors as lgf_plan_create; a problem's own error names the problem.
 */
lgf_status lgf_plan_create_multi(const int32_t *block_ijk, const int64_t *block_offsets,
                                 const int32_t *n_levels, int32_t n_problems, int32_t n_b,
                                 int32_t interp_order, int32_t precision, int32_t interp_mode,
                                 const lgf_plan_options *opts, lgf_plan *out);

/*
 * Plan statistics: the work of one solve (Sec. 3.2 counts for this block set).
 *   pairs[l]   level 0: near (block, block) pairs; level l >= 1: interaction-list
 *              (target, source) interval pairs; each costs NW complex products
 *   intervals[l], groups[l]   intervals and sibling groups per level
 *   nw[l]      frequencies per spectrum at level l (0 where l has no products)
 *   top_product_level  highest level with a non-empty interaction list
 *   merged_level01     1 if levels 0 and 1 share one product pass (nw[1] is
 *                      then the level-0 spectrum size)
 *   n_problems         independent problems in the plan (lgf_plan_create_multi)
 *   persistent_ctas    CTAs (one per SM) of the persistent level-0 products, 0 if
 *                      that level uses another form
 *   n_levels           the largest level count of its problems
 *   fft_kernel         the level-0 FFT form in use (see lgf_plan_options)
 *   compensated_interp 1 if the CUDA-core Reg/Interp passes sum with
 *                      compensation (mode COMPENSATED, or NATIVE in a deep
 *                      FP32 plan), else 0
 */
#define LGF_MAX_LEVELS 24
typedef struct {
    int64_t n_points, n_blocks;
    int32_t n_levels, top_product_level, fft_size_level0, fft_size_interval;
    int64_t pairs[LGF_MAX_LEVELS + 1];
    int64_t intervals[LGF_MAX_LEVELS + 1];
    int64_t groups[LGF_MAX_LEVELS + 1];
    int64_t nw[LGF_MAX_LEVELS + 1];
    int64_t workspace_bytes;
    int32_t merged_level01;
    int32_t n_problems;
    int32_t persistent_ctas;
    int32_t fft_kernel;
    int32_t compensated_interp;
} lgf_plan_stats;

lgf_status lgf_plan_get_stats(lgf_plan plan, lgf_plan_stats *stats);

/* Device bytes the plan holds (workspace plus its share of cached spectra);
 * what a serving loop charges against its HBM budget. */
lgf_status lgf_plan_workspace_bytes(lgf_plan plan, size_t *bytes);

/* Points (n_blocks * n_b^3) of the plan. */
lgf_status lgf_plan_points(lgf_plan plan, int64_t *n_points);

/*
 * lgf_solve - u = G * f on the plan's blocks (Sec. 3.1 Steps 1-3).
 *   f_dev   device pointer, n_points values of the plan precision (read only)
 *   u_dev   device pointer, n_points values (written in full, never read);
 *           must not overlap f_dev
 *   stream  a cudaStream_t (NULL = legacy default stream)
 * Asynchronous on stream; every kernel of the solve runs on it.
 */
lgf_status lgf_solve(lgf_plan plan, const void *f_dev, void *u_dev, void *stream);

/*
 * lgf_solve_batch - n independent solves issued back to back on one stream.
 * plans[i] / f_dev[i] / u_dev[i] as for lgf_solve; the plans must be distinct.
 */
lgf_status lgf_solve_batch(const lgf_plan *plans, const void *const *f_dev,
                           void *const *u_dev, int32_t n, void *stream);

/*
 * Batches: many independent solves launched together (batched serving of
 * uneven problems).  lgf_batch_create records n (plan, f, u) triples; each
 * lgf_batch_launch forks the stream into a pool of up to 16 streams, runs the
 * solves round-robin on the pool so they overlap on the device, and joins the
 * pool back into the stream.  use_graph = 1 captures the whole batch once
 * into a CUDA graph (after one uncaptured warm-up solve of every plan, during
 * lgf_batch_create) and each launch replays it.
 *   plans      n distinct plans (all on the current device); the batch keeps
 *              pointers to them: destroy the batch before its plans
 *   f_dev[i], u_dev[i]  device buffers of plan i, fixed for the batch's life
 * A batch must not be launched again before its previous launch finished
 * (the plans' workspaces are reused).
 */
typedef struct lgf_batch_s *lgf_batch;
lgf_status lgf_batch_create(const lgf_plan *plans, const void *const *f_dev, void *const *u_dev,
                            int32_t n, int32_t use_graph, lgf_batch *out);
lgf_status lgf_batch_launch(lgf_batch batch, void *stream);
lgf_status lgf_batch_destroy(lgf_batch batch);

/*
 * lgf_selftest_bounded_wait - diagnostic of the bounded device waits (no
 * counterpart in the paper).  The library's kernels never spin without a
 * limit: a wait that runs out sets a status word and the kernel returns, so
 * a stalled producer turns into an error code instead of a hang.  This call
 * runs one such wait on an mbarrier phase: complete != 0 completes the phase
 * (returns LGF_OK); complete == 0 leaves it pending, so the wait gives up
 * after limit_us microseconds of the GPU's global timer and the call returns
 * LGF_ERR_TIMEOUT with the context still usable.
 *   limit_us   1 .. 2000000
 * Synchronous (device-wide synchronize).
 */
lgf_status lgf_selftest_bounded_wait(int32_t complete, int32_t limit_us);

/*
 * lgf_measure_fma_peak - measured arithmetic peak of the current device (no
 * counterpart in the paper: the denominator of the rooflines of the products
 * and transforms, which run on the CUDA cores' fused multiply-add pipes).
 * Every SM runs as many CTAs as fit, each thread 16 independent chains of
 * fused multiply-adds; CUDA events time each launch; flop = 2 per FMA lane.
 *   kind         0 = fma.rn.f64, 1 = fma.rn.f32, 2 = fma.rn.f32x2 (two FP32
 *                lanes per instruction)
 *   reps         1..100 timed launches after one warm-up; the best is kept
 *   flops_per_s  receives the best launch's rate
 *   ms           receives that launch's duration
 * Synchronous on the legacy default stream; allocates a small buffer.
 */
lgf_status lgf_measure_fma_peak(int32_t kind, int32_t reps, double *flops_per_s, double *ms);

/*
 * lgf_solve_host - lgf_solve with host buffers: copies f to the plan's device
 * staging buffer, solves, copies u back, and waits for the stream.
 *   f_host, u_host  host pointers of n_points values (pinned memory is faster)
 */
lgf_status lgf_solve_host(lgf_plan plan, const void *f_host, void *u_host, void *stream);

/*
 * lgf_solve_host_pipelined - n_steps solves of one plan from host buffers,
 * the copies overlapped with the solves inside the library (end-to-end
 * throughput of a stream of inputs).  Step k copies f_host[k] into one of two
 * plan-owned device input buffers on a library-owned host-to-device stream,
 * solves on `stream` once that copy landed and the same buffer pair's
 * previous result has left, and copies the result into u_host[k] on a
 * library-owned device-to-host stream; so step k + 1's input copy and step
 * k - 1's result copy run while step k solves.
 *   f_host, u_host  n_steps host pointers each (pinned memory lets the copies
 *                   overlap; pointers may repeat), n_points values per buffer
 *   n_steps         >= 0
 *   stream          the solves' stream; the first copy waits for the work
 *                   already queued on it
 * Returns when every result is in host memory.  The staging buffers (four
 * field-sized device arrays) are allocated at the first call and kept.
 */
lgf_status lgf_solve_host_pipelined(lgf_plan plan, const void *const *f_host, void *const *u_host,
                                    int32_t n_steps, void *stream);

/* Waits for the plan's last solve (the last one not captured into a graph)
 * and reports any asynchronous error; other work on the device is not waited
 * for. */
lgf_status lgf_plan_sync(lgf_plan plan);

/*
 * Per-kernel timing (tracing).  lgf_plan_set_timing(plan, capacity) makes the
 * next solves bracket each kernel launch by a CUDA event pair on the solve's
 * stream, for up to `capacity` launches in total (0 turns it off).
 * lgf_plan_timings waits for those events and returns, per kernel name, the
 * summed elapsed time and the number of launches, then starts a new tally.
 *   names               max_kernels x 32 chars (NUL-terminated names)
 *   total_ms, count     max_kernels entries
 *   n_kernels           receives the number of distinct names (may exceed max)
 *   launches_per_solve  receives the kernel launches of the last solve (or NULL)
 */
lgf_status lgf_plan_set_timing(lgf_plan plan, int32_t capacity);
lgf_status lgf_plan_timings(lgf_plan plan, int32_t max_kernels, int32_t *n_kernels, char *names,
                            double *total_ms, int32_t *count, int32_t *launches_per_solve);

/*
 * lgf_conv_blocks - the FFT convolution of isolated blocks (the special case
 * of Sec. 4.2, "FFT Conv.": the whole active grid is one block, and the method
 * reduces to one zero-padded FFT convolution, Eqs. alg_upfft, alg_mult,
 * alg_dwfft): u_b = G * f_b over block b alone, for every block b, in one
 * kernel launch.  A CTA takes a block through the forward transform, the
 * product with the block's own kernel spectrum and the inverse transform with
 * the spectrum in shared memory (it never reaches device memory); the results
 * equal those of a one-block plan and of lgf_solve_blocks_noalloc.
 *
 *   f_dev, u_dev  device pointers, n_blocks * n_b^3 values of the precision,
 *                 block-major with x fastest (as lgf_solve); f_dev == u_dev
 *                 (in place) is allowed, any other overlap of the two byte
 *                 ranges is LGF_ERR_INVALID_ARG
 *   n_blocks      1 .. 2^31 - 1
 *   n_b           4, 8 or 16 (else LGF_ERR_UNSUPPORTED); precision
 *                 LGF_FP32 or LGF_FP64
 *   stream        cudaStream_t; the launch is asynchronous
 *
 * The first call on a device for an (n_b, precision) computes the kernel
 * spectrum (FP64 on the host), allocates it on the device and uploads it with
 * a synchronous copy (it stays until the process exits); make that first call
 * before any stream capture.  Errors: LGF_ERR_OOM if that allocation fails,
 * LGF_ERR_CUDA for a launch failure.
 */
lgf_status lgf_conv_blocks(const void *f_dev, void *u_dev, int64_t n_blocks, int32_t n_b, int32_t precision,
                           void *stream);

/*
 * lgf_solve_blocks_noalloc - solves every block as its own isolated problem,
 * u_b = G * f_b over block b alone (each block is a separate one-block domain,
 * as lgf_solve computes for a one-block plan), without allocating any device
 * memory.  The paper has no counterpart: this exists for callers that cannot
 * call cudaMalloc while they run (allocator hooks, loops whose memory was
 * fixed up front, frameworks that own the device heap).
 *
 * All working memory (block spectra, kernel spectra, item tables) lives in one
 * file-scope device array of 32 MiB that every GPU loading the library holds
 * until the process exits.  The first call on a device, with that device
 * current, looks up the array's device address and uploads the tables and
 * the kernel spectra of every (n_b, precision) pair with synchronous copies;
 * make that first call before any stream capture.  Later calls only launch
 * kernels on the stream.
 *
 *   f_dev, u_dev  device pointers, n_blocks * n_b^3 values of the precision,
 *                 block-major with x fastest (as lgf_solve); the two byte
 *                 ranges must not overlap (LGF_ERR_INVALID_ARG)
 *   n_blocks      1 .. lgf_noalloc_max_blocks(n_b, precision); more is
 *                 LGF_ERR_INVALID_ARG (232 for n_b = 16 in FP32, 116 in FP64)
 *   n_b           4, 8 or 16;  precision  LGF_FP32 or LGF_FP64
 *   stream        cudaStream_t; asynchronous after the first call
 *
 * Every call shares the array and it keeps the last call's contents; each
 * call writes all it reads.  Calls that overlap on the GPU (other streams or
 * host threads) race on the array and must be serialised by the caller.
 */
lgf_status lgf_solve_blocks_noalloc(const void *f_dev, void *u_dev, int64_t n_blocks, int32_t n_b,
                                    int32_t precision, void *stream);
lgf_status lgf_noalloc_max_blocks(int32_t n_b, int32_t precision, int64_t *max_blocks);

/* Frees the plan and its workspace.  Returns without waiting: the workspace
 * comes from the stream-ordered allocator and is released once the plan's
 * last solve has completed, so destroying an idle plan does not stall other
 * work on the device.  A plan whose solves were captured into a graph must
 * outlive every launch of that graph (lgf_batch_destroy waits for them). */
lgf_status lgf_destroy(lgf_plan plan);

/* Message for the calling thread's last failed call ("" if none). */
const char *lgf_last_error(void);

/*
 * Host-side pieces of the plan builder, exposed for checking.
 *
 * lgf_green_values - G(n) of the 7-point Laplacian (App. A, Eq. lgf3) in FP64
 *   for n triples (n x 3 int32, any signs) into out (n doubles); host only.
 * lgf_interp_weights - the 1D interpolation matrices W[c][i][p], c = 0, 1 (2 x
 *   (n_b+1) x (n_b+1) doubles): weight of parent node p for node i of child c
 *   (Sec. 2.5 with the nearest-n_max rule); Reg applies the transpose.
 */
lgf_status lgf_green_values(const int32_t *n, int64_t count, double *out);
lgf_status lgf_interp_weights(int32_t n_b, int32_t n_max, double *W);

/*
 * Choice of the interpolation parameters for a target error (Sec. 2.5, the
 * two-step procedure; host only).
 *
 * lgf_lebesgue_constant - Lambda_n of n equally spaced nodes: the maximum
 *   over their interval of sum_i |l_i(x)| (l_i the Lagrange basis), which
 *   bounds how much interpolation amplifies perturbations of the nodal
 *   values (Eq. leb).  1 <= n <= 40.
 *
 * lgf_select_interp - Step 1: n_max = the largest node count n with
 *   Lambda_n^3 eps_p < eps (tensor-product interpolation in 3D; eps_p the
 *   unit roundoff of the precision, 2^-53 FP64, 2^-24 FP32), n <= 17.
 *   Step 2: the smallest supported block size n_b (4, 6, ..., 32; n_I = n_b + 1
 *   >= n_max) whose interpolation of the field the method interpolates errs
 *   by less than eps relative to the field: the LGF of the nearest sources a
 *   parent interval's interaction list can hold (on the face of the interval
 *   one interval width away: its corners, edge midpoints and centre),
 *   interpolated from the parent's nodes (spacing 2) to its children's nodes
 *   (spacing 1) with the n_max stencil.
 *     eps          target relative error, 0 < eps < 1
 *     precision    LGF_FP32 or LGF_FP64 (sets eps_p)
 *     n_max, n_b   receive the choice (interp_order = n_max - 1)
 *     lebesgue     receives Lambda_{n_max} (may be NULL)
 *     interp_err   receives the step-2 error of the chosen n_b (may be NULL)
 *   LGF_ERR_UNSUPPORTED when no supported block size reaches eps; the outputs
 *   then hold the largest size tried and its error.
 */
lgf_status lgf_lebesgue_constant(int32_t n, double *out);
lgf_status lgf_select_interp(double eps, int32_t precision, int32_t *n_max, int32_t *n_b, double *lebesgue,
                             double *interp_err);

#ifdef __cplusplus
}
#endif
#endif /* LGF_H */
