/*
 * fst.h -- C ABI of libfst: GB300-native (sm_103a) evaluation and randomized
 * least-squares core refit of functional sparse Tucker (FST) models.
 *
 * Paper: P. Rai, H. Kolla, L. Cannada, A. Gorodetsky, "Randomized Functional
 * Sparse Tucker Tensor for Compression and Fast Visualization of Scientific
 * Data", arXiv 1907.05884.
 *
 * Conventions (all entry points):
 *   - Plain C types only.  Pointers documented "device" must be CUDA device (or
 *     managed) memory of the current device; "host" pointers are ordinary CPU memory.
 *   - The caller owns every point, value, index and output buffer.  The library
 *     owns fst_model objects and the scratch memory it keeps inside them.
 *   - Work is enqueued on the given stream (0 = legacy default stream).  Calls
 *     documented "asynchronous" return before the GPU finishes; the others end
 *     with a synchronisation of that stream because they return host results.
 *   - Errors are returned as fst_status, never thrown; fst_last_error() gives a
 *     thread-local message for the last failing call of the calling thread.
 *   - Points are structure-of-arrays: xyz[0..n) = y1, xyz[n..2n) = y2,
 *     xyz[2n..3n) = y3.  Points outside the model box are evaluated by polynomial
 *     extrapolation (no clamping).
 *   - Limits: 1 <= r_k <= FST_MAX_RANK, 0 <= p_k <= FST_MAX_DEGREE.
 *   - One model may be evaluated from several host threads and streams at once.  A call
 *     that changes a model's core (fst_refit*, fst_model_set_core) must not overlap, on
 *     the host or on the GPU, evaluations of that model: order them (the same stream, or
 *     an event).  Tensor-core operand images of a changed core are rebuilt by the next
 *     evaluation after a device synchronisation, so no kernel still reads a buffer that
 *     is being rewritten.
 */
#ifndef FST_H
#define FST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FST_MAX_RANK 32
#define FST_MAX_DEGREE 127
#define FST_MAX_WAVELET_LEVEL 6       /* 2^s <= 64 cells */
#define FST_MAX_WAVELET_DEGREE 15

typedef struct fst_model fst_model;            /* opaque, device-resident, owned by the library */
typedef struct CUstream_st* fst_stream;        /* a cudaStream_t */

typedef enum {
    FST_OK = 0,
    FST_EINVAL = -1,        /* bad argument (null pointer, size, rank, degree) */
    FST_ENOMEM = -2,        /* device or host allocation failed */
    FST_ECUDA = -3,         /* a CUDA runtime call failed; see fst_last_error() */
    FST_ENOTSPD = -4,       /* normal matrix not positive definite (rank-deficient sample) */
    FST_ERANK = -5,         /* fewer sampled rows than unknowns (m < R) */
    FST_ETIMEOUT = -6,      /* a bounded device wait gave up */
    FST_EFORMAT = -7,       /* model file malformed */
    FST_ENOTCONV = -8,      /* iterative refinement did not converge */
    FST_EUNSUPPORTED = -9   /* precision or shape not supported by this build */
} fst_status;

/* Arithmetic of the contraction / Gram assembly.  FP64 and FP32 run on the CUDA
 * cores; TF32, BF16 and BF16X3 (A = A_hi + A_lo split, three products) run the
 * contraction on the tcgen05 tensor cores with FP32 accumulation. */
typedef enum { FST_FP64 = 0, FST_FP32 = 1, FST_TF32 = 2, FST_BF16 = 3, FST_BF16X3 = 4 } fst_prec;

/* Host description of a model with d = 3 (Sec. 2, eq. func_tuck and eq. sparse).
 *   r[k]      Tucker rank of mode k.
 *   p[k]      maximum Legendre degree of mode k (p[k]+1 basis functions).
 *   lo, hi    the box mapped affinely onto [-1,1]^3.
 *   colptr[k] (r[k]+1 entries), rowidx[k], val[k]: column j of mode k holds the
 *             degrees n (0 <= n <= p[k], strictly increasing within a column) and
 *             coefficients W^k_{n,j} of the orthonormal Legendre functions
 *             phi_n(t) = sqrt(2n+1) L_n(t), i.e. w^(k)_j(t) = sum_n W^k_{n,j} phi_n(t).
 *   alpha     core, r1*r2*r3 values in C order [j1][j2][j3].
 * All host pointers; fst_model_create copies them. */
typedef struct {
    int32_t r[3];
    int32_t p[3];
    double lo[3];
    double hi[3];
    const int32_t* colptr[3];
    const int32_t* rowidx[3];
    const double* val[3];
    const double* alpha;
} fst_model_desc;

/* ---------------------------------------------------------------- models */

/* Copy a host description to the current device (synchronous).  Fails with
 * FST_EINVAL on out-of-range ranks/degrees or unsorted/out-of-range degrees. */
fst_status fst_model_create(const fst_model_desc* desc, fst_model** out);

/* Free a model and its scratch (synchronises the device first).  NULL is a no-op. */
void fst_model_free(fst_model* model);

/* Shape: ranks, degrees and stored coefficients per mode.  Any output may be NULL. */
fst_status fst_model_shape(const fst_model* model, int32_t r[3], int32_t p[3], int32_t nnz[3]);

/* Copy the model back to caller-owned host buffers sized from fst_model_shape:
 * colptr[k] (r[k]+1), rowidx[k] and val[k] (nnz[k]), alpha (r1 r2 r3), lo/hi (3).
 * Any pointer may be NULL to skip that part.  Synchronous. */
fst_status fst_model_read(const fst_model* model, int32_t* colptr[3], int32_t* rowidx[3],
                          double* val[3], double* alpha, double lo[3], double hi[3]);

/* Replace the core with r1 r2 r3 host values (C order).  Synchronous. */
fst_status fst_model_set_core(fst_model* model, const double* alpha);

/* Factor functions in a multiwavelet space (Sec. 4.2, Algorithm 1's choice between the
 * Legendre space and a multiresolution space per singular vector, Fig. 3).  W_{s,q} is the
 * space of piecewise polynomials of degree <= q on the 2^s equal cells of each box axis,
 * with the orthonormal multiresolution basis (inner product 1/2 int f g over [-1, 1]):
 * function n = 0..q is phi_n on the whole axis; function (q+1)(2^l + c) + i is the wavelet
 * psi_{l,c,i}(t) = 2^{l/2} psi_i(2^l (t+1) - 2c - 1) on cell c of level l (l < s, i <= q),
 * where psi_0..psi_q are sgn(t) phi_i(t) orthonormalised in order against phi_0..phi_q and
 * the earlier psi.  A coordinate y is in finest cell f when f of the interior boundaries
 * lo + ((hi - lo) c) 2^-s, c = 1..2^s-1, are <= y (exact FP64 comparison of y); points
 * outside the box continue the first or last cell's polynomial.
 *   level, degree  s (0..FST_MAX_WAVELET_LEVEL) and q (0..FST_MAX_WAVELET_DEGREE), with
 *                  (q+1) 2^s <= 256
 *   col_wavelet[k] r[k] flags (host); column j of mode k with a nonzero flag holds, in
 *                  desc->rowidx / val, indices (0 <= idx < (q+1) 2^s, strictly increasing)
 *                  and coefficients of the functions of W_{s,q}; the other columns are
 *                  Legendre columns as in fst_model_desc.  col_wavelet[k] may be NULL
 *                  (no wavelet columns in mode k).
 * fst_model_create_wavelet copies everything like fst_model_create; the evaluators, refits,
 * fits and model files handle such models.  The factor-step tensor-core evaluator serves
 * Legendre-only models; wavelet models take the variant with factor values on the CUDA
 * cores.  FST_EINVAL on out-of-range parameters or indices. */
typedef struct {
    int32_t level;
    int32_t degree;
    const uint8_t* col_wavelet[3];
} fst_wavelet_desc;

fst_status fst_model_create_wavelet(const fst_model_desc* desc, const fst_wavelet_desc* wav, fst_model** out);

/* The model's multiwavelet space and column flags: *level = -1 when no column uses one
 * (then *degree = 0 and the flags are all 0).  col_wavelet[k] (r[k] bytes, host) may be
 * NULL.  Any pointer may be NULL. */
fst_status fst_model_read_wavelet(const fst_model* model, int32_t* level, int32_t* degree,
                                  uint8_t* col_wavelet[3]);

/* Binary model file (".fstm", little-endian): magic "FSTM", version, ranks,
 * degrees, box, CSC coefficients and the core, all values FP64. */
fst_status fst_model_save(const fst_model* model, const char* path);
fst_status fst_model_load(const char* path, fst_model** out);

/* ---------------------------------------------------------------- evaluation */

/* u~(y) at n points (Sec. 6: reconstruction is the evaluation of the basis
 * functions at the points of interest; eq. func_tuck).  xyz: device, 3n floats
 * SoA; out: device, n floats.  prec selects the contraction arithmetic: FST_FP32 on
 * CUDA cores, or FST_TF32 / FST_BF16 / FST_BF16X3 with the core contraction on the
 * tcgen05 tensor cores (factor values in FP32, FP32 accumulation).  Asynchronous and
 * allocation-free once the model is prepared (see fst_eval_prepare). */
fst_status fst_eval(const fst_model* model, const float* xyz, int64_t n, float* out,
                    fst_prec prec, fst_stream stream);

/* One evaluation instance of a batch: a model, its points (device, 3n floats SoA) and
 * its output (device, n floats). */
typedef struct {
    const fst_model* model;
    const float* xyz;
    int64_t n;
    float* out;
} fst_eval_item;

/* Evaluate many instances -- different models, uneven ranks and point counts -- with one
 * persistent launch per size class of ranks (tensor-core precisions): the items are cut
 * into runs of 128-point tiles, about four runs per SM; with several instances the blocks
 * of the factor-step evaluator take runs in order from a counter (otherwise the runs are
 * split over the blocks by estimated cost), and a block reloads a model's core tiles only
 * when the instance changes.  Every result equals the single-instance fst_eval of that item bit for bit.
 * FST_FP32 runs one CUDA-core launch per item.  items: host array; a model must not be
 * refitted while it is being evaluated.  Asynchronous: the work lists go through a
 * per-device ring of 8 pinned/device staging slots that only grow (the ninth call in
 * flight waits for the first); models not yet prepared for prec are prepared first
 * (synchronously). */
fst_status fst_eval_batched(const fst_eval_item* items, int32_t count, fst_prec prec, fst_stream stream);

/* A prepared batch (the persistent batched launch): the items' work lists and size classes
 * are built and uploaded once; fst_eval_plan_run then only launches (one persistent kernel
 * per size class of ranks), allocates nothing and does not synchronise, so it can be
 * captured into a CUDA graph and replayed.  The models' cores and the items' buffers must
 * stay as they were when the plan was made (a refit changes the core: make a new plan).
 * Runs of one plan on different streams are ordered on the device (they share the plan's
 * run counters); inside a stream capture that ordering is the graph's.  Tensor-core
 * precisions only. */
typedef struct fst_eval_plan fst_eval_plan;
fst_status fst_eval_plan_create(const fst_eval_item* items, int32_t count, fst_prec prec,
                                fst_eval_plan** out);
fst_status fst_eval_plan_run(const fst_eval_plan* plan, fst_stream stream);
void fst_eval_plan_free(fst_eval_plan* plan);   /* waits for the device (cudaFree) */

/* Build, ahead of time, what fst_eval needs for a tensor-core precision (the core as
 * tensor-core operand tiles; rebuilt after the core changes), autotuning the model's size
 * class first if this device has not measured it (see fst_eval_autotune).  fst_eval does
 * the image build itself on first use with a synchronous upload; call this first to keep
 * fst_eval free of allocation and synchronisation.  Synchronous. */
fst_status fst_eval_prepare(fst_model* model, fst_prec prec);

/* Autotuner of the tensor-core evaluator.  For BF16 / BF16X3 two kernels can serve a model:
 * factor values on the CUDA cores (FP32) with the core contraction on the tensor cores, or
 * factor values on the tensor cores too (Legendre tiles x factor coefficients, BF16x3
 * products; degrees below 64).  Per device and size class (precision, rank bound, r3
 * padding, Legendre K) the library keeps the variant measured fastest; fst_eval_prepare
 * measures a class the first time it sees it, and fst_eval, fst_eval_batched and plans use the
 * table (an unmeasured class takes the tensor-core factor step where it is possible).
 * fst_eval_autotune measures the model's class now on n_probe points of its box (one warm-up
 * and three timed runs per variant, CUDA events), records the faster and returns the mean
 * times (ms; both -1 when only the CUDA-core factor step can serve the class: nothing is
 * timed) and the choice (0: factor values on the CUDA cores, 1: on the tensor cores).
 * Synchronous.  fst_eval_autotune_set records a
 * choice by hand (-1 forgets the class). */
fst_status fst_eval_autotune(fst_model* model, fst_prec prec, int64_t n_probe, fst_stream stream,
                             float* ms_cuda_core_factors, float* ms_tensor_core_factors, int32_t* choice);
fst_status fst_eval_autotune_set(const fst_model* model, fst_prec prec, int32_t choice);

/* Report (and clear) a bounded device wait that expired inside a tensor-core evaluation
 * on this device since the last check: FST_ETIMEOUT, else FST_OK.  Synchronises stream. */
fst_status fst_eval_check(fst_stream stream);

/* The same in FP64 throughout (device xyz: 3n doubles, out: n doubles).  Asynchronous. */
fst_status fst_eval_f64(const fst_model* model, const double* xyz, int64_t n, double* out,
                        fst_stream stream);

/* Points of an axis-aligned slice -- the 2D visualisation query of Sec. 6 (Fig. 6) --
 * written into a device buffer: the plane y_axis = value, the two other axes sampled on a
 * res0 x res1 node grid spanning [lo, hi] (both ends included; the lower-numbered free
 * axis varies slowest).  xyz: device, 3 * res0 * res1 floats, SoA.  Asynchronous. */
fst_status fst_slice_points(int32_t axis, double value, const double lo[3], const double hi[3],
                            int32_t res0, int32_t res1, float* xyz, fst_stream stream);

/* ---------------------------------------------------------------- sampling */

/* Uniform sample of m distinct rows of [0,Q) without replacement (Algorithm 2,
 * sampling step): row q gets the key splitmix64(seed, q) -- the (q+1)-th output
 * of a splitmix64 stream seeded with `seed` -- and the m rows with the smallest
 * keys are written to idx (device, m int64) in ascending order.  m >= Q gives
 * every row.  Asynchronous; uses model-free scratch owned by the library. */
fst_status fst_sample_rows(uint64_t seed, int64_t Q, int64_t m, int64_t* idx, fst_stream stream);

/* The paper has no counterpart to this entry point: it is a service for callers
 * that must not allocate device memory -- for example an in-situ visualisation
 * hook running inside a simulation whose own pool already owns the device memory,
 * or a latency-bound loop that cannot absorb the implicit device synchronisation
 * of cudaMalloc.  It returns exactly what fst_sample_rows returns, but calls no
 * cudaMalloc, cudaFree or other allocating routine: its scratch (520 KiB)
 * is one fixed device array inside libfst that every GPU which loads the library
 * keeps until the process exits.
 *   - Limit: Q <= 2^29 rows; larger Q returns FST_EINVAL (use fst_sample_rows).
 *   - The first call on each device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any stream
 *     capture.
 *   - All calls share the one array (the selection state and histogram are
 *     cleared at the start of each call): calls that overlap on the GPU -- on two
 *     streams, or from two threads -- race and may return wrong rows.  Order them
 *     on one stream or synchronise between them.
 * idx: device, m int64 (caller-owned).  Asynchronous. */
fst_status fst_sample_rows_static(uint64_t seed, int64_t Q, int64_t m, int64_t* idx, fst_stream stream);

/* ---------------------------------------------------------------- refit */

typedef struct {
    int32_t max_refine;       /* refinement (preconditioned CG) steps after the first solve (default 32) */
    double refine_tol;        /* stop when the CG step is <= tol ||alpha|| (default 1e-13 FP64, 1e-8 else) */
    int32_t fp64_cholesky;    /* 1: factor the normal matrix in FP64 (default: FP64 only for FST_FP64) */
} fst_refit_opts;

typedef struct {
    int64_t m;                /* rows used */
    int32_t refine_steps;     /* refinement steps taken */
    int32_t fallback_fp64;    /* 1 if the FP32 factorisation failed and FP64 was used */
    int32_t fallback_bf16x3;  /* 1 if a TF32 / BF16 Gram failed to factor and the BF16x3 Gram was used */
    int32_t shifted_preconditioner; /* 1 if the factor is of G + 2^-12 diag(G) (G too ill-conditioned
                                       for an FP32 factorisation; the CG still solves G) */
    double first_rel_change;  /* ||alpha_refined - alpha_first|| / ||alpha_refined|| */
    double last_rel_update;   /* ||delta|| / ||alpha|| of the last step */
    double ms_sample, ms_factors, ms_gram, ms_cholesky, ms_refine;   /* GPU time per phase */
} fst_refit_report;

/* Re-estimate the core by least squares over sampled rows of the original data
 * (Sec. 5, eq. rand_core; Algorithm 2 with uniform sampling of S = m > R rows,
 * without the sign-flip/mixing steps): draws idx with fst_sample_rows(seed),
 * forms the normal equations G = A^T A, h = A^T b over the Khatri-Rao rows
 * a_q = w1(y1_q) (x) w2(y2_q) (x) w3(y3_q) in `prec`, factors G by Cholesky and
 * refines alpha by conjugate gradients on the normal equations preconditioned by
 * that factor, with A p and A^T q accumulated in FP64.  If the FP32 factorisation of a
 * TF32 / BF16 Gram fails, the BF16x3 Gram is factored; if that fails, G + 2^-12 diag(G);
 * then everything is redone in FP64.
 * xyz (3Q floats SoA), u (Q floats): device.  idx: device int64 rows to use, or
 * NULL to draw m rows with `seed`.  opts, report: host, may be NULL.  On success
 * the model's core is replaced.  Synchronous (returns host status).
 * FST_ERANK if m < R, FST_ENOTSPD if G is not positive definite in FP64. */
fst_status fst_refit(fst_model* model, const float* xyz, const float* u, int64_t Q,
                     const int64_t* idx, int64_t m, uint64_t seed, fst_prec prec,
                     const fst_refit_opts* opts, fst_refit_report* report, fst_stream stream);

/* One refit instance of a batch: a model (each item a different model), its points (device,
 * 3Q floats SoA) and values (device, Q floats), and the rows to draw (fst_sample_rows with
 * `seed`, m >= R). */
typedef struct {
    fst_model* model;
    const float* xyz;
    const float* u;
    int64_t Q;
    int64_t m;
    uint64_t seed;
} fst_refit_item;

/* Refit many models (Sec. 5, eq. rand_core; Algorithm 2 per item) -- uneven ranks and point
 * counts -- concurrently: `streams` (1..64) worker
 * host threads, each with its own non-blocking CUDA stream of the current device, take the
 * items in order and run fst_refit on them, so the launches of different instances overlap on
 * the GPU (small instances do not fill it alone).  Every result equals that of fst_refit on
 * the item (the same kernels, rows and arithmetic).  reports: host array of count entries, or
 * NULL.  The inputs must be complete when the call starts (its streams do not wait on any of
 * the caller's).  Synchronous: returns after every refit has finished; on failure returns the
 * status of the first failed item (the others still ran).  Two items naming one model: EINVAL. */
fst_status fst_refit_batched(const fst_refit_item* items, int32_t count, fst_prec prec,
                             const fst_refit_opts* opts, int32_t streams, fst_refit_report* reports);

/* Refit many models (Sec. 5, eq. rand_core; Algorithm 2 per item) with shared launches, on
 * one stream.  Per item: the rows (fst_sample_rows with the item's seed), the factor values,
 * A^T b and the Gram in `prec`.  Then the FP32 factorisations of all items run as one
 * schedule, every launch doing the same panel step for each matrix that still has it; and the
 * preconditioned conjugate gradients of all items advance together, one launch per step for
 * every item (per rank class r3 <= 8 / 16 / 24 / 32 where a kernel is specialised), the
 * triangular solves of all items in one launch per direction.  Small instances, which leave
 * most of the GPU idle alone and are bound by their chains of short launches, then share
 * those launches.  Each item's arithmetic is that of fst_refit, so every core equals
 * fst_refit's on the item bit for bit; an item whose factorisation fails or whose iteration
 * does not converge is redone alone by the fst_refit procedure (with its fallbacks), as is
 * every item when opts asks for the FP64 factorisation.  items: host array (the
 * fst_refit_batched item; one model per item); reports: host array of count, or NULL (for a
 * grouped item, ms_cholesky and ms_refine are those of the whole group).  The items' data
 * must be ready in `stream`'s order.  Synchronous; returns the status of the first failed
 * item after all items have run (the others' cores are replaced). */
fst_status fst_refit_grouped(const fst_refit_item* items, int32_t count, fst_prec prec,
                             const fst_refit_opts* opts, fst_refit_report* reports, fst_stream stream);

/* Algorithm 2 with its mixing step (Sec. 5): the core minimising || S F D W alpha - S F D u ||
 * over all Q points, W the Khatri-Rao rows of the points (eq. rand_core), D = diag(+-1) with
 * D_q = -1 when bit 63 of the splitmix64 key of row q under seed_signs is set, F the
 * normalised Walsh-Hadamard transform over the rows padded with zeros to N = 2^ceil(log2 Q)
 * (the paper asks for a fast orthonormal mixing; this is the real one taken), and S the m rows
 * of fst_sample_rows(seed_rows, N, m).  Mixing spreads the row leverage scores, so uniform
 * sampling sees every direction of the design.  FP64 throughout, solved by the normal
 * equations (Cholesky); F D W is materialised (N (R + 1) doubles of device memory), so this is
 * for problems of that size.  xyz: device, 3Q doubles SoA; u: device, Q doubles; R <= m <= N
 * (FST_ERANK below R).  Synchronous; the model's core is replaced. */
fst_status fst_refit_mixed(fst_model* model, const double* xyz, const double* u, int64_t Q, int64_t m,
                           uint64_t seed_signs, uint64_t seed_rows, fst_refit_report* report, fst_stream stream);

/* The normal equations of the sampled problem alone (eq. rand_core restricted to the
 * rows idx): G = A^T A (device, R x R FP32 row-major; the lower triangle is written,
 * the upper triangle is unspecified) with A_{s,(i,j,k)} = w1_i w2_j w3_k at the points
 * of rows idx (device, m int64), assembled in `prec` (FP32 on CUDA cores; TF32, BF16,
 * BF16X3 on tensor cores with FP32 accumulation), and, if h is not NULL, h = A^T b
 * (device, R doubles) with b = u[idx].  Synchronous for tensor-core precisions. */
fst_status fst_normal_matrix(const fst_model* model, const float* xyz, const float* u, int64_t Q,
                             const int64_t* idx, int64_t m, fst_prec prec, float* G, double* h,
                             fst_stream stream);

/* The factorisation step of the refit on its own: G = L L^T in place for an R x R
 * row-major FP32 symmetric positive definite matrix (device).  The lower triangle is read
 * and overwritten by L; the strict upper triangle is left as it was.  128-wide panels:
 * diagonal blocks and panel solves in FP32 on the CUDA cores; trailing updates on the
 * tcgen05 tensor cores in BF16x3 (each L entry split into BF16 high and low parts, three
 * products, FP32 accumulation), so L has relative errors near 1e-5: in the refit it is the
 * preconditioner of the conjugate gradients, which set the final accuracy.  Synchronous;
 * allocates and frees its scratch.  FST_ENOTSPD if a pivot is at or below
 * 16 eps_32 max_i G_ii. */
fst_status fst_cholesky_f32(float* G, int32_t R, fst_stream stream);

/* Fault-injection hook for tests (the paper has no counterpart): the clock-cycle budget of
 * the bounded spin waits of the one-launch triangular solves (refit, its conjugate
 * gradients) on the current device, for calls made after this one; 0 restores the default
 * (about one second).  A budget of a few cycles makes a solve block give up on a value the
 * previous block row has not published yet: the block records the expiry in the solve's
 * error word and finishes, and the refit returns FST_ETIMEOUT without touching the model;
 * the device context stays usable.  The waits are plain loads, with no asynchronous copies
 * or tensor-core work in flight, so an expiry leaves nothing behind.  FST_EINVAL for
 * cycles < 0.  Not thread-safe with respect to refits running on the device. */
fst_status fst_set_wait_limit(int64_t cycles);

/* FP64 refit (xyz 3Q doubles, u Q doubles; FP64 Gram, FP64 Cholesky). */
fst_status fst_refit_f64(fst_model* model, const double* xyz, const double* u, int64_t Q,
                         const int64_t* idx, int64_t m, uint64_t seed,
                         const fst_refit_opts* opts, fst_refit_report* report, fst_stream stream);

/* ---------------------------------------------------------------- construction */

/* Parameters of the construction (Algorithm 1 and Sec. 4).  Limits: 2 <= grid[k] <= 256,
 * 1 <= max_rank[k] <= FST_MAX_RANK, 0 <= max_degree <= 63. */
typedef struct {
    int32_t grid[3];          /* interpolation grid: grid[k] equispaced nodes on [-1,1], both ends included */
    double sample_frac;       /* fraction of the Q points splatted onto the grid, in (0, 1] */
    double eps;               /* ST-HOSVD precision: per mode, discarded eigenvalues sum to <= eps^2 ||U||^2 / 3 */
    int32_t max_rank[3];      /* rank caps (the rank is also at most grid[k]) */
    int32_t max_degree;       /* Legendre degree p of every mode (p + 1 candidate functions per column) */
    int32_t fixed_rank;       /* 1: r_k = min(max_rank[k], grid[k]) instead of the eps rule */
    double oversample;        /* refit rows m = min(ceil(oversample * R), Q) */
    uint64_t seed;            /* interpolation subset: fst_sample_rows(seed); refit rows: seed + 0x632BE59BD9B4E019 */
    const double* grid_values;/* host, optional: grid[0]*grid[1]*grid[2] values (C order) that replace the
                                 interpolation step (sample_frac is then ignored) */
    int32_t wavelet;          /* 1: also fit every column in W_{wav_level, wav_degree} (fst_wavelet_desc) and
                                 keep the fit with the smaller leave-one-out error; 0: Legendre only */
    int32_t wav_level;        /* s, with (wav_degree + 1) 2^s <= 64 */
    int32_t wav_degree;       /* q */
} fst_fit_params;

typedef struct {
    int32_t r[3];             /* Tucker ranks of the model (after dependent functions are dropped) */
    int32_t r_hosvd[3];       /* ranks chosen by the ST-HOSVD */
    int32_t nnz[3];           /* stored Legendre coefficients per mode */
    int32_t fill_sweeps;      /* Jacobi sweeps needed to fill the empty grid nodes */
    int32_t eig_sweeps[3];    /* Jacobi eigensolver sweeps per mode */
    int64_t n_interp;         /* points splatted onto the grid */
    int64_t m;                /* rows of the core refit */
    double compression_ratio; /* Q / (R + nnz): values only, positions not counted (Sec. 2, Table 2) */
    double ms_interp, ms_hosvd, ms_sparse, ms_refit;   /* GPU time per step */
    fst_refit_report refit;
    int32_t n_wavelet[3];     /* kept columns in the multiwavelet space, per mode */
} fst_fit_report;

/* Optional host outputs of the intermediate steps; any pointer may be NULL.
 *   grid_values  grid[0]*grid[1]*grid[2]: the filled grid tensor U (C order)
 *   eigvals[k]   grid[k]: eigenvalues of the mode-k Gram matrix of the partially reduced
 *                tensor, descending
 *   W[k]         grid[k] * max_rank[k] (capacity): the kept eigenvectors, grid[k] x r[k]
 *                row-major, each with its largest-magnitude entry positive
 *   core_hosvd   max_rank product (capacity): the ST-HOSVD core, r1 r2 r3 values
 *   col_nnz      r1 + r2 + r3 (capacity, mode-major): coefficients kept per column
 *   col_loo      r1 + r2 + r3 (capacity): leave-one-out error of the chosen support
 *   col_kept     r1 + r2 + r3 (capacity): 1 if the fitted function was kept, 0 if dropped
 *   col_wavelet  r1 + r2 + r3 (capacity): 1 if the column's fit is in W_{s,q}, 0 if in P_p
 *   col_loo_alt  r1 + r2 + r3 (capacity): leave-one-out error of the other space's fit
 *                (only with params->wavelet)
 * (r here: the ST-HOSVD ranks) */
typedef struct {
    double* grid_values;
    double* eigvals[3];
    double* W[3];
    double* core_hosvd;
    int32_t* col_nnz;
    double* col_loo;
    int32_t* col_kept;
    int32_t* col_wavelet;
    double* col_loo_alt;
} fst_fit_trace;

/* Build a model from Q scattered values (Algorithm 1, then the core refit of Algorithm 2):
 *   1. fst_sample_rows(seed) draws ceil(sample_frac Q) points; each is splatted onto the
 *      8 nodes of its grid cell with trilinear weights and a node takes the weighted mean;
 *      empty nodes are filled by Jacobi sweeps (an empty node takes the mean of its filled
 *      6-neighbours of the previous sweep) -- the paper's linear interpolation to a grid
 *      (Sec. 4.1);
 *   2. ST-HOSVD of the grid tensor at precision eps (Sec. 4.1): modes 1, 2, 3 in order, the
 *      eigenvectors of the FP64 mode Gram matrix (parallel cyclic Jacobi);
 *   3. each factor column gets a sparse orthonormal-Legendre expansion: the Lasso-LARS path
 *      on the grid nodes, every visited support refitted by least squares and the one with
 *      the least leave-one-out error kept (Sec. 3, Sec. 4.2); with params->wavelet the same
 *      fit in W_{s,q} too, and the column keeps the space whose fit has the smaller
 *      leave-one-out error (within 1e-12 mean(y^2) of each other: Legendre; Algorithm 1's
 *      basis choice); a fitted function in the span of the earlier ones of its mode
 *      (relative residual <= 1e-6, in-order Gram-Schmidt on the coefficients, or with
 *      wavelets on exact quadrature samples of the functions) is dropped, so the refit
 *      below has independent columns;
 *   4. fst_refit of the core on m = min(ceil(oversample R), Q) rows drawn with
 *      seed + 0x632BE59BD9B4E019, in `prec` (FST_FP64: the points are widened to FP64 and
 *      fst_refit_f64 runs).
 * Steps 1-3 are FP64.  xyz (3Q floats SoA), u (Q floats): device.  lo, hi: host box mapped
 * onto [-1,1]^3 (NULL: [-1,1]).  opts, trace, report: host, may be NULL.  On success *out
 * is a new model owned by the caller (fst_model_free).  Synchronous.
 * FST_EINVAL if no grid node receives a sample; refit errors as fst_refit. */
fst_status fst_fit(const float* xyz, const float* u, int64_t Q, const double lo[3], const double hi[3],
                   const fst_fit_params* params, fst_prec prec, const fst_refit_opts* opts,
                   fst_fit_trace* trace, fst_fit_report* report, fst_model** out, fst_stream stream);

/* ---------------------------------------------------------------- order-4 models */

/* Models of order 4 (eq. func_tuck with d = 4: three space axes and time, the SP4D case of
 * Sec. 6 and Table 1), f(y) = sum alpha_{j1 j2 j3 j4} w1_{j1}(y1) w2_{j2}(y2) w3_{j3}(y3)
 * w4_{j4}(y4), each factor function a sparse combination of the orthonormal Legendre
 * functions of the coordinate mapped to [-1,1] by the model's box (eq. sparse).  Ranks up to
 * FST4_MAX_RANK a mode (the paper's SP4D ranks are 30 x 38 x 5 x 11), degrees up to
 * FST_MAX_DEGREE, r1 r2 r3 r4 <= 2^24.  Evaluation runs on the CUDA cores. */
#define FST4_MAX_RANK 64
typedef struct fst_model4 fst_model4;
typedef struct {
    int32_t r[4];
    int32_t p[4];
    double lo[4], hi[4];
    const int32_t* colptr[4];   /* host CSC of each mode, as fst_model_desc */
    const int32_t* rowidx[4];
    const double* val[4];
    const double* alpha;        /* host, r1 r2 r3 r4 values, C order [j1][j2][j3][j4] */
} fst_model4_desc;
/* Copies the description to the device.  Synchronous.  *out: fst_model4_free. */
fst_status fst_model4_create(const fst_model4_desc* desc, fst_model4** out);
void fst_model4_free(fst_model4* model);
/* The core (host, r1 r2 r3 r4 doubles, C order). */
fst_status fst_model4_read_core(const fst_model4* model, double* alpha);
/* f at n points (device, 4n values SoA: x[0..n) = y1, ..., x[3n..4n) = y4) into out (device,
 * n values): FP32 or FP64 arithmetic on the CUDA cores.  Asynchronous. */
fst_status fst_eval4(const fst_model4* model, const float* x, int64_t n, float* out, fst_stream stream);
fst_status fst_eval4_f64(const fst_model4* model, const double* x, int64_t n, double* out, fst_stream stream);
/* The core refit (Sec. 5, eq. rand_core; Algorithm 2 with uniform sampling): m rows drawn by
 * fst_sample_rows(seed, Q, m), factor values in FP64 rounded to FP32; the normal matrix
 * G = A^T A of the rows (w1 (x) w2) (x) (w3 (x) w4) from the packed Khatri-Rao operand on the
 * tensor cores in `prec` (TF32, BF16 or BF16X3; G and its saved copy / transpose take 8 R^2
 * bytes of device memory, 31 GB at R = 62,700, besides the packed operand of a row block), its FP32
 * Cholesky factor (G is the FP32 sum of the Grams of blocks of 16,384 rows: the tensor cores'
 * FP32 sums over all m rows at once round at about 1e-3 of the largest diagonal entry at
 * R = 62,700; if G still does not factor, that of G + delta diag(G), delta 2^-12 .. 2^-2, which
 * preconditions the unshifted equations; report->shifted_preconditioner is the step of delta
 * taken), alpha_0 = G^-1 A^T b,
 * then conjugate gradients on A^T A alpha = A^T b preconditioned by the factor, with A p and
 * A^T q applied in the four-way factored form (FP32 products, FP64 sums) -- as fst_refit.
 * opts: max_refine steps (default 200), refine_tol (default 1e-8; the iteration also stops
 * when the update stops shrinking below 1e-6).  x (4Q floats SoA), u (Q floats):
 * device.  report: host, may be NULL.  Synchronous; on success the core is replaced.
 * R <= 131072; FST_ERANK if m < R, FST_ENOMEM if G does not fit, FST_ENOTSPD if no Gram
 * factors, FST_ENOTCONV if the iteration does not converge. */
fst_status fst_refit4(fst_model4* model, const float* x, const float* u, int64_t Q, int64_t m, uint64_t seed,
                      fst_prec prec, const fst_refit_opts* opts, fst_refit_report* report, fst_stream stream);

/* ---------------------------------------------------------------- errors */

const char* fst_status_str(fst_status s);
const char* fst_last_error(void);
/* Library build description (arch, version) -- a static string. */
const char* fst_build_info(void);
/* Number of CUDA kernels libfst has launched in this process (all devices). */
uint64_t fst_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif
