/*
 * bispec.h - C ABI of the GB300 (sm_103a) FFT bin-averaged 3D bispectrum estimator.
 *
 * The estimator is the fast bispectrum estimator (FBE) of Shaw et al., "A fast estimator
 * for quantifying the shape dependence of the 3D bispectrum" (arXiv:2107.14564), Sec. 2:
 *
 *   B(a,b,c) = V_c^3 sum_x d_a(x) d_b(x) d_c(x) / (V sum_x i_a(x) i_b(x) i_c(x))
 *
 * Eq. (2.7) with Eq. (2.10) (Ng^3 cancels), where for every spherical k shell n
 *   d_n(x) = sum_{k in n} F(k) e^{+i k.x}   (Eq. (2.8); D(k_n,x) = V_c d_n(-x))
 *   i_n(x) = sum_{k in n}      e^{+i k.x}   (Eq. (2.11))
 * and F(k) = sum_x delta(x) e^{-i k.x} is the unnormalised DFT of the density field
 * (Delta(k) = V_c F(k) is the Fourier transform of Eq. (2.1); V = L^3, V_c = (L/Ng)^3).
 * Bins are the shell triplets a >= b >= c with at least one closed triangle (Sec. 2.1),
 * labelled by (k1, mu, t) of Eq. (2.4).
 *
 * Conventions shared by every entry point
 *  - Grids are C-order [x][y][z]; z is the last axis, the axis the real FFT halves and the
 *    line of sight of the optional linear RSD factor (Eq. (3.4)).
 *  - A half spectrum is [Ng][Ng][Ng/2+1] interleaved complex (re, im): complex128 for
 *    BSP_FP64 plans, complex64 for BSP_FP32 and BSP_MIXED_BF16X3 plans. Index (i, j, l)
 *    holds the mode m = (i or i-Ng, j or j-Ng, l), the signed frequency below Ng/2.
 *  - Shell edges are in units of k_f = 2 pi / L. Mode m is in shell n iff
 *    e_n^2 <= |m|^2 < e_{n+1}^2 (integer |m|^2); k = 0 is in no shell.
 *  - No exception crosses the ABI. Every call returns a bsp_status; on failure
 *    bsp_last_error() gives a message (thread-local, valid until the next call on the
 *    same thread). A CUDA error inside a call is reported as BSP_ERR_CUDA.
 *  - The caller owns every buffer it passes. A plan owns its device tables, scratch and
 *    cached shell fields. A plan is not safe for concurrent use from several threads.
 *  - Calls taking a `stream` (a cudaStream_t, NULL = legacy default stream) enqueue their
 *    GPU work on it and return without waiting, unless documented otherwise.
 */
#ifndef BISPEC_H
#define BISPEC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BSP_API __attribute__((visibility("default")))
#else
#define BSP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BSP_OK = 0,
  BSP_ERR_INVALID_ARG = 1,   /* a null pointer, a size or an enum out of range */
  BSP_ERR_ALIASING = 2,      /* a shell reaches k >= 2 pi Ng / (3 L), the cap after Eq. (2.12) */
  BSP_ERR_OOM = 3,           /* a device or host allocation failed */
  BSP_ERR_CUDA = 4,          /* a CUDA runtime or launch error */
  BSP_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
  BSP_ERR_NOT_SUPPORTED = 6, /* a grid size or option the library does not handle */
  BSP_ERR_NUMERIC = 7        /* a triangle count came out non-integral (Eq. (2.10)) */
} bsp_status;

typedef enum {
  BSP_FP64 = 0,         /* FP64 shell FFTs and FP64 triple products */
  BSP_FP32 = 1,         /* FP32 shell FFTs; FP32 products on CUDA cores, FP64 across chunks */
  BSP_MIXED_BF16X3 = 2  /* FP32 shell FFTs; tcgen05 split-BF16 products (hi*hi + hi*lo + lo*hi),
                           FP32 accumulation in tensor memory over short voxel runs, FP64 across */
} bsp_precision;

typedef enum {
  BSP_LABEL_SHELL_MEAN = 0,    /* k1, k2, k3 of Eq. (2.4): the mean |k| of the modes of each shell */
  BSP_LABEL_TRIANGLE_MEAN = 1  /* the mean |k_a|, |k_b|, |k_c| over the bin's closed triangles (the
                                  bin's average triangle, Sec. 2.1), from FP64 sums of Eq. (2.10)
                                  with one counting field weighted by |k|; plan time only */
} bsp_label_k;

typedef struct {
  int ng;                  /* grid points per side; even, 16..1024, of the form 2^p or 3*2^p */
  double box_len;          /* L, the side of the periodic cube (any length unit) */
  int n_shells;            /* N_s >= 1 */
  const double* edges_kf;  /* host, N_s + 1 strictly increasing edges in units of k_f (Sec. 2.1) */
  int n_mu, n_t;           /* (mu, t) cells over [0.5, 1]^2 (the region of Eq. (2.2)), >= 1 each */
  int rsd;                 /* 1: multiply the spectrum by 1 + beta (k_z/|k|)^2 (Eq. (3.4)) */
  double beta;             /* linear RSD parameter beta_1 of Eq. (3.4) */
  int precision;           /* a bsp_precision */
  size_t mem_budget_bytes; /* 0: hold every shell field of an estimate at once (N_s S^3 reals on the
                              evaluation grid of side S, bsp_plan_grid). Otherwise the most bytes of
                              shell fields the plan may hold: when the fields exceed it, estimates,
                              plan-time counts and bsp_grad make the X and Y passes once and then
                              produce and reduce the fields one x-slab of the evaluation grid at a
                              time (the largest slab within the budget, sums added in FP64), on one
                              contraction level. The X/Y pass buffers are outside the budget. A
                              budget below one x-plane of all shells is BSP_ERR_INVALID_ARG;
                              BSP_MIXED_BF16X3 plans whose fields exceed it need an evaluation grid
                              of 128..1024 points of the form 2^p or 3*2^p (else
                              BSP_ERR_NOT_SUPPORTED) and then hold one slab of split fields, so
                              bsp_contract refuses them. Results equal the unbudgeted plan's up to
                              the order of the sums. */
  int autotune;            /* 1: at creation, time the tensor-core contraction of every level with
                              its voxels split over 1, 2 and 4 x (SM count) blocks per tile group and
                              keep the fastest (BSP_MIXED_BF16X3 plans; the split changes only the
                              order of the FP64 cross-block sums), and time the persistent Y and Z
                              FFT passes with grids of 1 .. 16 x (SM count) blocks and keep the
                              fastest (FP32 and mixed plans on the warp passes; the grid changes no
                              value). No counterpart in the paper. */
  int k1_merge;            /* (mu, t) cells span this many neighbouring k1 shells (Sec. 2.1, last
                              paragraph: merging adjacent bins); 0 or 1: one shell per cell group */
  int label_k;             /* a bsp_label_k: the lengths the labels (mu, t) are formed from */
  int dim;                 /* 0 or 3: an Ng^3 cube binned in spherical shells. 2: an Ng^2 square of
                              side L binned in annular rings (the 2D box of Sec. 2.1): ng even up
                              to 4096, spectrum [Ng][Ng/2 + 1] (the last axis halved), fields
                              [N_s][S][S], B = A_c^3 sum d d d / (A sum i i i) with the cell area
                              A_c = (L / Ng)^2 and A = L^2; BSP_FP64 or BSP_FP32 only, without RSD,
                              triangle-mean labels, memory budget, bsp_spectrum or bsp_grad. */
  int order;               /* 0 or 3: the bispectrum. 4: the binned 4-point sum (trispectrum) that
                              the FFT estimator extends to (Sec. 4: modes below 2 pi Ng / (4 L)):
                              bins a >= b >= c >= e that can close, value V_c^4 sum_x d_a d_b d_c d_e
                              / (V sum_x i_a i_b i_c i_e), N_tri the number of ordered closed
                              quadrilaterals; it keeps the disconnected part (modes cancelling in
                              pairs). BSP_FP64 or BSP_FP32, at most 16 shells, n_mu = n_t = 1, no
                              memory budget or triangle-mean labels; bsp_contract and bsp_grad
                              refuse it. */
} bsp_plan_desc;

/* One bin of triangles (Sec. 2.1): shells a >= b >= c and their labels (Eq. (2.4)). */
typedef struct {
  int a, b, c;         /* shell indices, a >= b >= c */
  int i_mu, i_t;       /* (mu, t) cell after clamping mu and t to [0.5, 1] */
  int inside;          /* 1 iff (mu, t) satisfies Eq. (2.2) */
  double ntri;         /* N_tri of Eq. (2.9)/(2.10), an integer, ordered triples */
  double tsum;         /* sum_x i_a i_b i_c = Ng^3 N_tri (FP64, as computed) */
  double k1, k2, k3;   /* lengths of sides a, b, c (units of k_f) per the plan's bsp_label_k */
  double mu, t;        /* Eq. (2.4), unclamped (NaN for order-4 bins) */
  int e;               /* order-4 bins: the fourth shell, a >= b >= c >= e; -1 otherwise */
  int reserved;
} bsp_triplet;

typedef struct bsp_plan bsp_plan;

/* Build the binning plan (Sec. 2.1) and the triangle counts N_tri of every bin (Eq. (2.10),
 * computed on the GPU in FP64 from the counting fields of Eq. (2.11)); keep the bins with
 * N_tri > 0. Synchronous: returns when the plan is ready. Allocates the plan's device memory
 * on the current CUDA device with cudaMalloc. Errors: BSP_ERR_INVALID_ARG (desc null or out of
 * range, edges not increasing, an empty shell), BSP_ERR_ALIASING (edge beyond the cap after
 * Eq. (2.12)), BSP_ERR_NOT_SUPPORTED (ng), BSP_ERR_OOM, BSP_ERR_CUDA, BSP_ERR_NUMERIC. These
 * argument checks run before any CUDA call, so they also work on a machine without a GPU.
 * `stream`: the stream the plan's kernels use during creation. *out is NULL on failure. */
BSP_API bsp_status bsp_plan_create(const bsp_plan_desc* desc, void* stream, bsp_plan** out);

/* Free a plan and all its device memory (synchronises the device first). NULL is a no-op. */
BSP_API bsp_status bsp_plan_destroy(bsp_plan* plan);

/* Sizes of a plan: kept bins, shells, bytes of one shell-field set, device bytes held. */
BSP_API bsp_status bsp_plan_info(const bsp_plan* plan, int* n_triplets, int* n_shells,
                         size_t* field_bytes, size_t* device_bytes);

/* The contraction levels of a plan (no counterpart in the paper): for level l < *n_levels
 * (ascending side), level_side[l] = its grid side g and blocks_mult[l] = the voxel blocks per
 * tensor-core tile group divided by the SM count (the autotuner's choice; 1 without it; 0 for a
 * level on the CUDA cores). Split-BF16 plans may have merged levels (a pair on a larger grid than
 * its smallest exact one). Arrays: host, at least max_levels entries each, may be NULL. */
BSP_API bsp_status bsp_plan_tuning(const bsp_plan* plan, int* n_levels, int* level_side, int* blocks_mult,
                                   int max_levels);

/* Where each kept bin is summed (no counterpart in the paper; for tests and profiling): for bin t
 * < n (the order of bsp_plan_triplets), level[t] = index of its contraction level (as in
 * bsp_plan_tuning) and slot[t] = for split-BF16 plans the tensor-core tile and pair slot of its
 * pair, (tile group x tiles per group + tile) x 64 + slot, else -1. Arrays: host, n entries each
 * (n = the plan's kept bins), may be NULL. Errors: BSP_ERR_INVALID_ARG for a NULL plan or n other
 * than the number of kept bins. */
BSP_API bsp_status bsp_plan_bin_levels(const bsp_plan* plan, int n, int* level, int* slot);

/* Side of the plan's evaluation grid, ng_eval <= ng. Every shell mode has |m_i| <= r - 1, so a
 * triple product of shell fields only holds wavevectors with |k_i| <= 3 (r - 1); summed over any
 * grid of side S > 3 (r - 1) it keeps only k = 0, exactly as the ng^3 grid of Eq. (2.7) does (the
 * plane-wave identity of Eq. (2.6) and the cap after Eq. (2.12)). The plan samples the shell
 * fields (Eq. (2.8), (2.11)) on the smallest such S it has kernels for and scales its sums by
 * (ng / S)^3; results are those of the ng^3 grid up to rounding. */
BSP_API bsp_status bsp_plan_grid(const bsp_plan* plan, int* ng_eval);

/* The kept bins, in ascending (a, b, c) order; the host table is owned by the plan. */
BSP_API bsp_status bsp_plan_triplets(const bsp_plan* plan, const bsp_triplet** table, int* n);

/* Shell fields, Eq. (2.8), sampled on the plan's evaluation grid (S = bsp_plan_grid):
 * fields_out[n][i][j][l] = d_n(x) at x = (i, j, l) L / S for n < N_s (device, caller-owned,
 * N_s * S^3 reals: double for BSP_FP64 plans, float otherwise). With rsd=1 the Kaiser factor of
 * Eq. (3.4) is applied to the spectrum first. spec: device half spectrum of the ng grid. */
BSP_API bsp_status bsp_shell_fields(bsp_plan* plan, const void* spec, void* fields_out, void* stream);

/* Triple-product sums, the numerator of Eq. (2.7): msum[t] = sum_x d_a d_b d_c over the ng^3 grid
 * for every kept bin t, from shell fields on the evaluation grid laid out as bsp_shell_fields
 * writes them (device, read-only, 16-byte aligned); computed as (ng / S)^3 times the sum over
 * the S^3 grid (bins whose triple products fit a coarser divisor grid g of S are summed on that
 * grid, sampled from the given fields, times (ng / g)^3). msum: device, n_triplets doubles. Uses
 * the plan's contraction (bsp_precision). */
BSP_API bsp_status bsp_contract(bsp_plan* plan, const void* fields, double* msum, void* stream);

/* The whole estimator on one field, Eqs. (2.7)-(2.11) and the (mu, t) map:
 *   b_triplet[t] = V_c^3 msum[t] / (V tsum[t])                        (device, n_triplets)
 *   b_grid[g][i_mu][i_t] = V_c^3 sum msum / (V sum tsum) over the kept bins whose k1 shell a has
 *   a / k1_merge = g in that cell (merged bins, Sec. 2.1 last paragraph); NaN where no bin falls
 *   (device, ceil(N_s / k1_merge) * n_mu * n_t; may be NULL). spec: device half spectrum,
 *   read-only. */
BSP_API bsp_status bsp_estimate(bsp_plan* plan, const void* spec, double* b_triplet, double* b_grid,
                        void* stream);

/* bsp_estimate from HOST buffers: copies the half spectrum host->device on `stream`, runs the
 * estimator and copies b_triplet (and b_grid if not NULL) back to the host. Only the modes the
 * shells can reach are copied and read: the box |m_x|, |m_y| <= r - 1, 0 <= m_z <= r - 1 of the
 * outermost shell (Sec. 2.1; bsp_plan_host_input_bytes gives its size), so spec_host's other
 * entries may hold anything. Pinned host memory gives asynchronous copies; the call
 * synchronises `stream` before it returns. */
BSP_API bsp_status bsp_estimate_host(bsp_plan* plan, const void* spec_host, double* b_triplet_host,
                             double* b_grid_host, void* stream);

/* Forward DFT of a real field on the modes the plan uses: spec_out[i][j][l] = sum_x delta(x)
 * e^{-i k.x} (the half-spectrum layout above, complex64, device, caller-owned) for every mode of
 * the ball covered by the shells; entries outside that ball are left untouched (bsp_estimate
 * never reads them). delta_x: device, float [ng][ng][ng]. This is the transform that takes a
 * density field delta(x) to the Delta(k) = V_c F(k) of Eq. (2.1). FP32 and mixed plans with ng =
 * 2^p or 3 * 2^p in [128, 1024]; else BSP_ERR_NOT_SUPPORTED. Asynchronous on `stream`. */
BSP_API bsp_status bsp_spectrum(bsp_plan* plan, const float* delta_x, void* spec_out, void* stream);

/* Adjoint of bsp_estimate: dl_ddelta[x][y][z] = dL/d delta(x) on the ng^3 grid (device, float,
 * caller-owned) for an upstream gradient dl_db[t] = dL/dB_t of the kept bins (device, doubles),
 * at the field whose half spectrum is `spec` (device, the input of bsp_estimate). B_t is trilinear
 * in the shell fields (Eq. (2.7), (2.8)), so
 *   dL/d delta(y) = sum_k [sum_n S_n(k) K(k) G^_n(k)] e^{+i k.y},
 *   G_n = sum_t dL/dB_t V_c^3 / (V T_t) (product of the bin's other two fields), one term per
 *   position of n in the bin, G^_n its forward DFT and K the Kaiser factor of Eq. (3.4).
 * Shell fields are recomputed (nothing is kept from a forward call); the first call allocates
 * the adjoint buffers (about two shell-field sets). FP32 and mixed plans whose grid sides are 2^p
 * or 3 * 2^p in [128, 1024]; else BSP_ERR_NOT_SUPPORTED. Asynchronous on `stream`. */
BSP_API bsp_status bsp_grad(bsp_plan* plan, const void* spec, const double* dl_db, float* dl_ddelta,
                            void* stream);

/* Many estimates in one call: bsp_estimate(plans[i], specs[i], b_triplet[i], b_grid[i]) for i < n,
 * enqueued in order on `stream` (b_grid may be NULL, or hold NULL entries). Plans may repeat and
 * may differ in grid size; estimates that share a plan run one after the other (they share its
 * buffers). Errors: those of bsp_estimate, for the first failing entry. */
BSP_API bsp_status bsp_estimate_batched(bsp_plan* const* plans, const void* const* specs, int n,
                                        double* const* b_triplet, double* const* b_grid, void* stream);

typedef struct bsp_batch bsp_batch;

/* Capture the same n estimates as one CUDA graph for repeated replay with bsp_batch_run: every
 * pointer passed here is baked into the graph and must stay valid (and keep its size) for the
 * batch's lifetime; each distinct plan first runs one estimate outside the capture (on `stream`,
 * synchronised). Plans must not have timing enabled. Errors: BSP_ERR_INVALID_ARG, BSP_ERR_CUDA. */
BSP_API bsp_status bsp_batch_create(bsp_plan* const* plans, const void* const* specs, int n,
                                    double* const* b_triplet, double* const* b_grid, void* stream,
                                    bsp_batch** out);

/* Replay a captured batch on `stream` (one graph launch for every kernel of every estimate). */
BSP_API bsp_status bsp_batch_run(bsp_batch* batch, void* stream);

/* Free a batch (not its plans or buffers). NULL is a no-op. */
BSP_API bsp_status bsp_batch_destroy(bsp_batch* batch);

/* Per-bin numerators of the last bsp_estimate on this plan, msum[t] = sum_x d_a d_b d_c, as a
 * device pointer owned by the plan (n_triplets doubles, valid until the next call on it). */
BSP_API bsp_status bsp_last_sums(const bsp_plan* plan, const double** msum);

/* Synchronise `stream` and report a device-side failure raised by an earlier call on this plan:
 * BSP_ERR_TIMEOUT if a bounded wait inside a kernel gave up (the call's results are invalid). The
 * plan's failure flag is cleared when it is reported, so a later check reports only failures of
 * calls made after this one. */
BSP_API bsp_status bsp_plan_check(bsp_plan* plan, void* stream);

/* Self-test of the failure path above (no counterpart in the paper): enqueue on `stream` one warp
 * that waits, through the tensor-core contraction's bounded mbarrier wait capped at 4096 polls,
 * on a barrier nothing arrives at; the wait runs out and raises this plan's failure flag, so the
 * next bsp_plan_check returns BSP_ERR_TIMEOUT (once). Nothing else is in flight in that kernel:
 * the context stays usable. Errors: BSP_ERR_INVALID_ARG (NULL plan), BSP_ERR_CUDA (launch). */
BSP_API bsp_status bsp_selftest_wait_timeout(bsp_plan* plan, void* stream);

/* Stages of one bsp_estimate, in launch order (for bsp_timing_read and bsp_plan_stage_work). */
enum {
  BSP_STAGE_XPASS = 0,    /* shell-masked C2C along x (Eq. (2.8)) */
  BSP_STAGE_YPASS = 1,    /* C2C along y */
  BSP_STAGE_ZPASS = 2,    /* C2R along z: the shell fields d_n(x) (with x-slabs: every slab's Z pass
                             and contraction) */
  BSP_STAGE_CONTRACT = 3, /* triple products sum_x d_a d_b d_c (Eq. (2.7) numerator) */
  BSP_STAGE_FINALIZE = 4, /* cross-block sums, B = V_c^3 M / (V T) and the (mu, t) cells */
  BSP_N_STAGES = 5
};

/* Start (enable=1) or stop (0) per-stage timing of bsp_estimate on this plan. While enabled,
 * each bsp_estimate records CUDA events between its stages on the call's stream, for at most
 * `max_calls` calls after the last enable (the events are created here, not during the calls).
 * Enabling resets the accumulated times. Errors: BSP_ERR_INVALID_ARG, BSP_ERR_CUDA. */
BSP_API bsp_status bsp_timing_enable(bsp_plan* plan, int enable, int max_calls);

/* Average milliseconds per recorded call of each stage (ms[BSP_N_STAGES]), the number of
 * recorded calls and the number of kernels those calls launched. Waits for the recorded events. */
BSP_API bsp_status bsp_timing_read(bsp_plan* plan, double* ms, int* n_calls, long long* n_launches);

/* Algorithmic work of one bsp_estimate per stage: bytes[s] that stage must move to or from
 * device memory (reads of the non-zero inputs it needs plus its outputs, each once) and
 * flops[s] of its arithmetic core (0 where it is negligible): for the contraction, one product
 * per pair and one multiply-add per bin and voxel on CUDA cores, or 3 x 2 x pairs x padded shell
 * columns x voxels for the split-BF16 tensor-core GEMM, each pair counted on its smallest exact
 * contraction level (a split-BF16 plan may contract a pair on a larger level where that is
 * faster; the extra work is not counted). Host-side, no GPU work. */
BSP_API bsp_status bsp_plan_stage_work(const bsp_plan* plan, double* bytes, double* flops);

/* Bytes bsp_estimate_host copies host->device per call (the spectrum box of the outermost shell). */
BSP_API bsp_status bsp_plan_host_input_bytes(const bsp_plan* plan, size_t* bytes);

/* Grids of the persistent Y and Z FFT passes the autotuner picked (0: as many blocks as fit). */
BSP_API bsp_status bsp_plan_pass_tuning(const bsp_plan* plan, int* y_blocks, int* z_blocks);

/* The x-slabs an estimate streams under mem_budget_bytes: slab_planes x-planes of the evaluation
 * grid per slab (the last one may be thinner) and n_slabs of them; 0 and 1 when the plan holds
 * all fields at once. */
BSP_API bsp_status bsp_plan_slabs(const bsp_plan* plan, int* slab_planes, int* n_slabs);

/* Limits of bsp_triple_sums_noalloc (its scratch array has a fixed size). */
#define BSP_NOALLOC_MAX_TRIPLETS 4096
#define BSP_NOALLOC_MAX_SHELLS 64
#define BSP_NOALLOC_MAX_BLOCKS 304

/* Triple-product sums that allocate nothing: msum[t] = sum_x d_a(x) d_b(x) d_c(x) for the bins
 * triplets[3t..3t+2] = (a, b, c), from FP32 fields[n][v] (n < n_shells, v < n_vox), the layout
 * bsp_shell_fields writes. The paper has no counterpart of this entry point; it serves callers
 * that cannot call cudaMalloc: code inside a framework whose allocator owns the whole device
 * memory budget (a raw cudaMalloc there escapes its accounting), or a loop that must never enter
 * the driver's allocator after set-up. It needs no plan. Its per-block partial sums live in one
 * static device array of BSP_NOALLOC_MAX_BLOCKS * BSP_NOALLOC_MAX_TRIPLETS doubles (9.5 MiB) that
 * every GPU loading this library keeps until the process exits; the first call on a device looks
 * up that array's address (make this first call before any stream capture). Each call writes
 * every scratch entry it later reads, so nothing needs clearing, but all calls share the array:
 * calls that overlap on the GPU (other streams, other threads) race and give wrong sums.
 * fields, triplets (int, 3 per bin), msum (n_triplets doubles): device pointers, caller-owned.
 * Errors: BSP_ERR_INVALID_ARG for NULL pointers, n_shells outside [1, BSP_NOALLOC_MAX_SHELLS],
 * n_triplets outside [1, BSP_NOALLOC_MAX_TRIPLETS] or n_vox < 1; BSP_ERR_CUDA. A bin whose shell
 * indices are not all in [0, n_shells) gets msum = NaN (the kernel checks every index before it
 * reads, so no memory outside the inputs is touched). Accumulates in FP32 over runs of 1024 voxels
 * and in FP64 across. */
BSP_API bsp_status bsp_triple_sums_noalloc(const float* fields, int n_shells, long long n_vox,
                                           const int* triplets, int n_triplets, double* msum,
                                           void* stream);

/* Message of the last failing call on this thread ("" if none). */
BSP_API const char* bsp_last_error(void);

/* Library version string. */
BSP_API const char* bsp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BISPEC_H */
