/*
 * ppd.h -- C ABI of libppd: the preconditioned primal-dual (PPD) solver for
 * radio-interferometric imaging on one GB300 (sm_103a).
 *
 * Method: Onose, Dabbech & Wiaux (2017), "An accelerated splitting algorithm
 * for radio-interferometric imaging: when natural and uniform weighting meet".
 * The library solves
 *     min_x ||Psi^dagger x||_1  s.t.  x >= 0,  ||Phi_j x - y_j||_2 <= eps_j  (all blocks j)
 * (Section 3, Eq. "split-min-problem" with W = I) by Algorithm 3, with the
 * data-fidelity prox taken in the metric U_j (Section 4.1, Algorithm 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns a status: PPD_OK (0) or a negative PPD_ERR_* code.
 *   No C++ exception and no abort crosses this boundary; ppd_last_error()
 *   gives a one-line message for the calling thread's last failure.
 * - Host buffers passed in are read during the call and never retained; the
 *   caller keeps ownership.  Host buffers passed out are written in full.
 * - Pointers named *_dev are caller-owned DEVICE memory, used on the given
 *   CUDA stream (cudaStream_t passed as void*; NULL = the context's own
 *   stream, so pass cudaStreamLegacy to mean the legacy default stream);
 *   the call only enqueues work and does not synchronise.
 * - The image is row-major n0 x n1 (n0 rows).  Complex arrays are
 *   interleaved (re, im).  Device arrays use the context's precision:
 *   float for PPD_FP32_FP64NORMS, double for PPD_FP64_PLAIN.
 * - Visibility order at the boundary is always the caller's order; the
 *   library sorts internally (see ppd_get_bins for the order it uses).
 * - Call order: ppd_create -> ppd_set_visibilities -> ppd_set_weights ->
 *   ppd_iterate / ppd_get_image / operators.  Out of order: PPD_ERR_NOT_READY.
 *   Calling ppd_set_visibilities or ppd_set_weights again resets the solver
 *   state to x = 0.
 * - A context is not thread-safe; use one context per host thread.
 * - A context lives on the device that was current at ppd_create.  Every
 *   entry point makes that device current while it runs and gives the
 *   caller's current device back on return; *_dev pointers and streams
 *   must belong to that device.
 */
#ifndef PPD_H
#define PPD_H

#include <stdint.h>

#if defined(__GNUC__)
#define PPD_API __attribute__((visibility("default")))
#else
#define PPD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PPD_OK                  0
#define PPD_ERR_INVALID_ARG    -1   /* bad pointer, size, shape or parameter */
#define PPD_ERR_OOM            -2   /* device allocation failed */
#define PPD_ERR_CUDA           -3   /* a CUDA runtime call failed */
#define PPD_ERR_NONFINITE      -4   /* NaN/Inf in a norm or the image */
#define PPD_ERR_TIMEOUT        -5   /* a bounded device wait gave up */
#define PPD_ERR_NOT_READY      -6   /* call order violated */
#define PPD_ERR_UNSUPPORTED    -7   /* size outside what this build handles */

/* precision (config.precision) */
#define PPD_FP64_PLAIN          0   /* every array and reduction in double, kernels launched one by one */
#define PPD_FP32_FP64NORMS      1   /* float arrays, double norms / bounds / stop tests, one CUDA graph per iteration */

/* Algorithm 2 start point (config.inner_init) */
#define PPD_INNER_WARM          0   /* previous iteration's prox output (P_B(z) on the first iteration) */
#define PPD_INNER_CURRENT       1   /* zbar^(0) = z */

/* estimate of ||U^{1/2} Phi||_S^2 for eta (config.norm_method) */
#define PPD_NORM_LANCZOS        0   /* largest eigenvalue of Phi^dagger U Phi by the Lanczos process */
#define PPD_NORM_POWER          1   /* power iteration on Phi^dagger U Phi */

/* Algorithm 2 iteration (config.inner_solver) */
#define PPD_INNER_FB            0   /* Algorithm 2 as printed: zbar <- P_B(zbar - mu U (zbar - z)) */
#define PPD_INNER_FISTA         1   /* the same step at an extrapolated point, FISTA t-sequence
                                       (Section 4.1: faster proximal gradient methods, Tseng 2008);
                                       identical to PPD_INNER_FB for n_itr <= 2 */

typedef struct ppd_ctx ppd_ctx;

/* Solver configuration.  ppd_config_default() fills the paper's values
 * (Section 5.1: tau = 0.49, lambda = 1, kappa = 1e-4, n_itr = 1, no
 * randomisation; Section 5: oversampling 2 per axis, 8 x 8 Kaiser-Bessel). */
typedef struct {
    int32_t  n0, n1;            /* image rows / columns: multiples of 16 in [16, 4096] whose
                                   doubles 2 n have no prime factor above 5 (powers of two
                                   above 4096 in FP64) */
    int32_t  oversample;        /* grid K = oversample * n per axis; must be 2 */
    int32_t  kernel_width;      /* interpolation support J; must be 8 */
    double   kb_beta;           /* Kaiser-Bessel shape; 0 => 2.34 * J */
    int32_t  n_blocks;          /* number of data blocks d >= 1 */
    int32_t  wavelet_levels;    /* SARA decomposition depth; must be 4 */
    int32_t  n_itr;             /* Algorithm 2 sub-iterations per PPD iteration, >= 1 */
    double   tau;               /* primal step (0.49) */
    double   lambda;            /* relaxation; must be 1 */
    double   kappa;             /* normalised soft-threshold (1e-4) */
    double   eta;               /* 0 => 1/||U^{1/2} Phi||_S^2 (norm_method) */
    double   zeta;              /* 0 => 1/||Psi||_S^2 = 1 */
    int32_t  precision;         /* PPD_FP64_PLAIN or PPD_FP32_FP64NORMS */
    int32_t  precond;           /* 1: PPD with U = inverse sampling density; 0: U = I (PD) */
    int32_t  inner_init;        /* PPD_INNER_WARM or PPD_INNER_CURRENT */
    int32_t  use_graph;         /* 1: replay each iteration from a captured CUDA graph */
    int32_t  tile;              /* gridding tile side T (16 or 32); 0 => 16 */
    int32_t  chunk;             /* max visibilities per gridding work item; 0 => 1024 */
    int32_t  power_iters;       /* cap on the operator applications of the norm estimate; 0 => 1000 */
    double   power_tol;         /* relative change of the estimate that stops it; 0 => 1e-10
                                   (Lanczos in FP32: at least 2e-6) */
    void    *stream;            /* cudaStream_t for all work; NULL => library-created stream */
    int32_t  inner_solver;      /* PPD_INNER_FB (default) or PPD_INNER_FISTA */
    /* Stopping tests ("until convergence" in Algorithms 2 and 3; the paper
     * gives no test, these are the library's readings, evaluated in FP64 on
     * the device in both precisions): */
    double   inner_tol;         /* Algorithm 2: a block stops at the first step t with
                                   ||zbar^t - zbar^(t-1)|| <= inner_tol ||zbar^t||, at most
                                   n_itr steps; 0 => always n_itr steps */
    double   stop_tol;          /* Algorithm 3: ppd_iterate returns early once the relative
                                   variation of x is < stop_tol and every block residual
                                   ||Phi_j xt - y_j|| <= stop_eps_factor eps_j; 0 => off */
    double   stop_eps_factor;   /* 0 => 1.005 */
    int32_t  stop_every;        /* test the rule after every stop_every-th iteration of a
                                   ppd_iterate call (one host synchronisation each); 0 => 1 */
    int32_t  grid_warps;        /* warps per gridding CTA: 4 or 8 in FP32 (4 only in FP64); 0 =>
                                   FP32: 8, or 4 when the gridding has more than 12 work items
                                   per SM; FP64: 4; ppd_autotune chooses it in FP32 */
    uint64_t seed;              /* start vector of the norm estimate: 0 => all ones; otherwise
                                   x_i = 0.5 + 2^-53 (s_i >> 11), s_i the SplitMix64 output
                                   for counter seed + (i + 1) * 0x9E3779B97F4A7C15 */
    int32_t  norm_method;       /* PPD_NORM_LANCZOS (default) or PPD_NORM_POWER */
    int32_t  launch_overlap;    /* 1: a kernel of the iteration may start while the one before it
                                   in its stream drains (programmatic dependent launch, compute
                                   capability 9.0 and later); 0 (default): every kernel waits for
                                   its predecessor to finish.  Results are the same either way. */
    int32_t  degrid_threads;    /* threads per degridding CTA: 128 or 256 in FP32 (256 only in
                                   FP64); 0 => 256; ppd_autotune chooses it in FP32 */
    int32_t  pad1;
} ppd_config;

/* Per-call statistics (ppd_iterate).  All norms are computed in double. */
typedef struct {
    int32_t  iters_done;        /* PPD iterations completed by this context so far */
    int32_t  status;            /* status of the call */
    double   rel_var;           /* ||x^(t) - x^(t-1)|| / ||x^(t)|| of the last iteration */
    double   snr_db;            /* 20 log10(||x0|| / ||x0 - x||) if ppd_set_ground_truth was called, else NaN */
    double   max_res_over_eps;  /* max_j ||Phi_j xt - y_j|| / eps_j at the last iteration's data step */
    double  *block_residual;    /* optional caller buffer of n_blocks doubles: ||Phi_j xt - y_j|| (whitened) */
    int32_t *inner_steps;       /* optional caller buffer of n_blocks int32: Algorithm 2 steps each
                                   block took in the last iteration (0: outside the active set) */
    int32_t  stopped;           /* 1 if the stop_tol rule ended the call before n_iters */
    int32_t  iters_run;         /* iterations this call ran */
} ppd_stats;

/* Parameters resolved by ppd_set_weights (and ppd_set_prior_weights /
 * ppd_reweight): zeta is the value the primal step uses, the configured zeta
 * divided by ||Psi W||_S^2. */
typedef struct {
    double   eta, zeta, tau, kappa;
    double   op_norm_sq;        /* ||U^{1/2} Phi||_S^2 (0 if eta was given) */
    int32_t  power_iters_done;  /* operator applications of the norm estimate */
    int32_t  K0, K1;            /* oversampled grid */
    int32_t  tile;              /* gridding tile side */
    int32_t  chunk;             /* max visibilities per work item */
    int64_t  n_chunks;          /* gridding work items */
    int64_t  M;                 /* visibilities */
    double   convergence_lhs;   /* tau*zeta*||Psi W||^2 + tau*eta*||U^{1/2}Phi||^2 (Eq. "convergence-req-explicit-pd"), < 1 */
    double   psiw_norm_sq;      /* ||Psi W||_S^2 of the prior weights (1 when W = I) */
    double   alpha;             /* clip level of the prior step, kappa * ||Psi W||_S^2 */
    int32_t  grid_warps;        /* warps per gridding CTA */
    int32_t  degrid_threads;    /* threads per degridding CTA */
} ppd_params;

/* Fill *cfg with the paper's defaults (n0 = n1 = 0 must still be set). */
PPD_API void ppd_config_default(ppd_config *cfg);

/* Create a context on the current CUDA device.  Validates cfg (sizes,
 * oversample = 2, J = 8, 4 levels, lambda = 1) and allocates the image-side
 * state (x, xt, the 9 SARA dual images u_i, the oversampled grids).
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
PPD_API int ppd_create(ppd_ctx **out, const ppd_config *cfg);

/* Free everything the context owns.  NULL is accepted. */
PPD_API void ppd_destroy(ppd_ctx *ctx);

/* Load the coverage and data (Section 2, Eq. "inverse-problem"; blocks as in
 * Section 3.1, Eq. "data-split").
 *   M         number of visibilities, 1 <= M < 2^31
 *   uv        M x 2 doubles, row-major: omega_m in [-pi, pi)^2 (radians per
 *             pixel); column 0 runs along image rows (axis 0)
 *   y         M x 2 doubles (re, im): raw, un-whitened visibilities
 *   block_id  M int32 in [0, n_blocks)
 * Bins every visibility on the oversampled grid (FP64, bit-exact), sorts them
 * into the library's processing order and counts visibilities per grid cell
 * (the sampling density used by the default preconditioner).
 * Errors: INVALID_ARG (NULL, M out of range, omega outside [-pi, pi], block
 * out of range, non-finite y), OOM, CUDA. */
PPD_API int ppd_set_visibilities(ppd_ctx *ctx, int64_t M, const double *uv, const double *y,
                         const int32_t *block_id);

/* Weights and bounds (Section 2: Theta; Section 4.3: U; Section 5.1: eps).
 *   theta  M doubles > 0, natural weights 1/sigma_e (NULL => all 1)
 *   U      M doubles > 0, preconditioner diagonal (NULL => 1/(visibilities in
 *          the visibility's nearest cell of the oversampled grid) when
 *          precond = 1, all 1 when precond = 0)
 *   eps    n_blocks doubles > 0, l2 bounds on the whitened residual of each
 *          block (NULL => sqrt(M_j + 2 sqrt(M_j)), two chi^2 standard
 *          deviations above its mean); ignored for blocks with no visibility
 * Then resolves eta (config.norm_method when config.eta = 0), mu_j =
 * 1/max(U_j)^2 (Algorithm 2) and resets the state to zero.
 * Errors: NOT_READY, INVALID_ARG, NONFINITE, OOM, CUDA. */
PPD_API int ppd_set_weights(ppd_ctx *ctx, const double *theta, const double *U, const double *eps);

/* Optional ground truth (n0*n1 doubles, row-major) for the SNR in ppd_stats
 * (Section 5: SNR = 20 log10(||x0|| / ||x0 - x||)).  NULL clears it. */
PPD_API int ppd_set_ground_truth(ppd_ctx *ctx, const double *x_true, int64_t len);

/* Run n_iters iterations of Algorithm 3 (lambda = 1, all blocks and bases
 * every iteration).  Work is enqueued on the context stream; if stats is
 * non-NULL the call synchronises and fills it.  n_iters >= 0.  With
 * config.stop_tol > 0 the call tests the global stopping rule (see
 * ppd_config) after every stop_every-th iteration, synchronising each time,
 * and returns as soon as it holds (stats->stopped = 1).
 * Errors: NOT_READY, INVALID_ARG, NONFINITE, TIMEOUT, CUDA. */
PPD_API int ppd_iterate(ppd_ctx *ctx, int32_t n_iters, ppd_stats *stats);

/* Copy the current image x^(t) to the host as n0*n1 doubles (synchronises).
 * len must equal n0*n1.  Errors: NOT_READY, INVALID_ARG, CUDA. */
PPD_API int ppd_get_image(ppd_ctx *ctx, double *x_out, int64_t len);

/* Resolved parameters (after ppd_set_weights). */
PPD_API int ppd_get_params(ppd_ctx *ctx, ppd_params *out);

/* Binning and ordering, for bit-exact checks (synchronises).  Each pointer
 * may be NULL.  All arrays have M entries in the CALLER's order except perm.
 *   perm     int64: perm[i] = caller index of the i-th visibility in the
 *            processing order (ascending tile of the centred grid, block,
 *            centred base row, centred base column, caller index)
 *   base0/1  int32: first interpolation tap (floor(kappa) - 3) mod K per axis,
 *            kappa = (omega * K) * 0.15915494309189535 in FP64
 *   count    int32: visibilities sharing the nearest cell
 *            (floor(kappa + 0.5) mod K per axis) */
PPD_API int ppd_get_bins(ppd_ctx *ctx, int64_t *perm, int32_t *base0, int32_t *base1, int32_t *count);

/* Autotuner for the gridding work decomposition: for each tile side
 * T in {16, 32} and work-item size C in {512, 1024, 2048} (visibilities per
 * CTA) it rebuilds the visibility order from the inputs of the last
 * ppd_set_visibilities / ppd_set_weights calls and, in FP32, tries gridding
 * warps per CTA in {4, 8} and degridding threads per CTA in {128, 256}; it
 * times `iters` PPD iterations of each candidate with CUDA events and keeps
 * the fastest; eta is kept, the solver state is reset to zero.  The chosen
 * tile and work-item size are returned (either pointer may be NULL);
 * ppd_get_params reports all four.
 * Errors: NOT_READY, INVALID_ARG, OOM, CUDA. */
PPD_API int ppd_autotune(ppd_ctx *ctx, int32_t iters, int32_t *tile_out, int32_t *chunk_out);

/* Solver state for checkpoint / resume and warm starts (Algorithm 3 takes
 * and returns x, xt, u_i, v_j; Algorithm 1 restarts Algorithm 3 from them):
 * a self-describing blob holding x, xt, the 9 dual images u_i, the data
 * duals v, the warm start p of Algorithm 2 (processing order), the per-block
 * flags of which blocks have been active (randomised active sets) and the
 * iteration count, tagged with the precision, sizes and a fingerprint of the
 * visibility order.  ppd_get_state with blob = NULL sets *bytes to the size
 * needed; otherwise *bytes must be at least that size and the blob is
 * written (synchronises).  ppd_set_state accepts only a blob made by a
 * context with the same precision, sizes and visibility order; resuming from
 * it reproduces an uninterrupted run bit for bit.
 * Errors: NOT_READY, INVALID_ARG (size, tag or fingerprint mismatch), CUDA. */
PPD_API int ppd_get_state(ppd_ctx *ctx, void *blob, int64_t *bytes);
PPD_API int ppd_set_state(ppd_ctx *ctx, const void *blob, int64_t bytes);

/* Re-weighted l1 (Section 3.2, Algorithm 1, Eq. "reweighting").  The prior
 * weights W_i are diagonal, one value per SARA coefficient, stored like the
 * 9 dual images u_i: 9 * n0 * n1 values, basis-major (Dirac, db1 .. db8),
 * each basis in the Mallat quadrant layout of ppd_psi_analysis.  With W set,
 * the prior step of Algorithm 3 becomes u_i <- clip(u_i + W_i Psi_i^dagger xt,
 * alpha), ut_i = Psi_i W_i u_i, with alpha = kappa ||Psi W||_S^2 and the primal
 * step uses zeta / ||Psi W||_S^2 (so the convergence condition keeps its
 * value); ||Psi W||_S^2 comes from a power iteration on Psi W^2 Psi^dagger
 * (start all-ones, cfg power_iters / power_tol).  The solver state (x, xt,
 * u, v) is kept, so the next ppd_iterate warm-starts from it as Algorithm 1
 * asks.  Weights persist across ppd_set_weights and ppd_set_state; they are
 * not part of the state blob.  A ppd_group holding the context re-captures
 * its graph on its next ppd_group_iterate.
 *
 * ppd_set_prior_weights: w = host array of len = 9 n0 n1 doubles, finite and
 *   >= 0, copied; w = NULL restores W = I.  Synchronises.
 * ppd_reweight: W = omega / (omega + |Psi^dagger x|) from the current primal
 *   iterate x, computed on the device (Eq. "reweighting"); omega > 0.
 *   Algorithm 1's schedule is omega^(k) = 0.25^k omega^(0), omega^(0) = 1e-2
 *   (Section 5.1).  Synchronises.
 * ppd_get_prior_weights: host copy (FP64) of W, all ones when W = I.
 * Errors: INVALID_ARG (NULL, len, negative or non-finite weight, omega),
 * NONFINITE (||Psi W|| zero or not finite: the context is left with W = I),
 * OOM, CUDA. */
PPD_API int ppd_set_prior_weights(ppd_ctx *ctx, const double *w, int64_t len);
PPD_API int ppd_reweight(ppd_ctx *ctx, double omega);
PPD_API int ppd_get_prior_weights(ppd_ctx *ctx, double *w, int64_t len);

/* Randomised active sets (Algorithm 3, "generate sets P and D"; Section 4.2:
 * only the dual variables in the sets are updated; Section 4.4: the sets are
 * drawn with nonzero probabilities, independently and identically along the
 * iterations).  Queues the sets of the next n_iters iterations:
 *   blocks  host array n_iters x n_blocks bytes, row t = the set D of the
 *           t-th next iteration (nonzero = data block j updated), or NULL
 *           (every block, every iteration)
 *   bases   host array n_iters x 9 bytes, row t = the set P (Dirac, db1 ..
 *           db8; nonzero = basis i updated), or NULL (every basis)
 * Both are copied.  A block outside D keeps v_j and its Algorithm 2 warm
 * start (its gridded contribution is reused without recomputation); a basis
 * outside P keeps u_i.  A block that has never been active starts
 * Algorithm 2 from P_B(z), as every block does on the first iteration.  The
 * rows are consumed one per iteration by ppd_iterate and ppd_group_iterate;
 * once they are used up every set is full until the next call.  n_iters = 0
 * drops the queue and returns to the plain iteration.  The draws are the
 * caller's (e.g. Bernoulli masks from a seeded generator); the queue position
 * is not part of the state blob.  Synchronises.
 * Errors: INVALID_ARG (NULL context, n_iters < 0), OOM, CUDA. */
PPD_API int ppd_set_active_sets(ppd_ctx *ctx, int32_t n_iters, const uint8_t *blocks, const uint8_t *bases);

/* Phi x = Theta G F Z x (Section 2): x_dev n0*n1 reals -> y_dev M complex
 * (caller order, whitened by theta).  Enqueued on stream.  Uses the
 * context's internal grid, so it must not overlap ppd_iterate on the same
 * context.  Errors: NOT_READY, INVALID_ARG, CUDA. */
PPD_API int ppd_op_forward(ppd_ctx *ctx, const void *x_dev, void *y_dev, void *stream);

/* Phi^dagger y = Re(Z^T F^H G^H Theta^H y): y_dev M complex (caller order)
 * -> x_dev n0*n1 reals.  Same rules as ppd_op_forward. */
PPD_API int ppd_op_adjoint(ppd_ctx *ctx, const void *y_dev, void *x_dev, void *stream);

/* Batched independent problems (the paper's problems are independent once
 * their data are fixed; the batch fills the GPU with several of them).  A
 * group holds n FP32 contexts that have weights set; ppd_group_iterate
 * advances every one of them by n_iters iterations of Algorithm 3, each
 * iteration of the whole group being one launch of a CUDA graph captured from
 * all the contexts' kernels on their own streams.  Results are identical to
 * iterating each context alone.  The contexts must not be used elsewhere
 * while the group runs; destroy the group before its contexts.
 * Errors: INVALID_ARG (NULL, n < 1, FP64 context, per-kernel timing on),
 * NOT_READY (a context without weights), CUDA. */
typedef struct ppd_group ppd_group;
PPD_API int ppd_group_create(ppd_group **out, ppd_ctx *const *ctxs, int32_t n);
PPD_API int ppd_group_iterate(ppd_group *g, int32_t n_iters);
PPD_API void ppd_group_destroy(ppd_group *g);

/* Phi^dagger without allocating: the same result as ppd_op_adjoint (same
 * arguments, layouts and stream rules), for callers that cannot let the
 * library allocate device memory during the call, such as applications with a
 * fixed device-memory budget reserved at start-up or real-time loops that must
 * not block on the allocator or meet an out-of-memory error mid-way.  The
 * paper has no counterpart; this is a deployment variant of the operator.
 * The gridding scratch (one (T+8)^2 complex tile per work item, see
 * ppd_params.n_chunks) comes from one fixed device array of
 * PPD_NOALLOC_SCRATCH_BYTES that the library holds on every GPU it is loaded
 * on until the process exits.  The call runs on the context's device (see
 * the conventions above) and uses that device's copy of the array.  The
 * first call on a device looks up that array's device address, so make the
 * first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU race and give
 * wrong results.  No cudaMalloc, cudaFree or other allocating routine is
 * called.  Errors: NOT_READY, INVALID_ARG, UNSUPPORTED (scratch needed above
 * the fixed size), CUDA. */
#define PPD_NOALLOC_SCRATCH_BYTES (32u << 20)
PPD_API int ppd_op_adjoint_noalloc(ppd_ctx *ctx, const void *y_dev, void *x_dev, void *stream);

/* Psi^dagger x (Section 2.2, Section 5.1: Dirac + db1..db8, 4 levels,
 * periodic, Mallat layout, each basis scaled by 1/3): x_dev n0*n1 reals ->
 * c_dev 9*n0*n1 reals (basis-major).  Enqueued on stream. */
PPD_API int ppd_psi_analysis(ppd_ctx *ctx, const void *x_dev, void *c_dev, void *stream);

/* Psi c = (1/3) sum_i Psi_i c_i: c_dev 9*n0*n1 reals -> x_dev n0*n1 reals. */
PPD_API int ppd_psi_synthesis(ppd_ctx *ctx, const void *c_dev, void *x_dev, void *stream);

/* Per-kernel timing with CUDA events on the context stream.  enable = 1
 * records an event pair around every kernel the iteration launches (inside
 * the captured graph too) and runs the iteration's two independent branches
 * one after the other, so each pair brackets one kernel only (the iteration
 * is then slower than with timing off); ppd_timing_collect() adds the durations of the
 * launches completed since the last collect (synchronises) to running sums;
 * ppd_timing_read() returns, for up to n kernel names, the summed
 * milliseconds and launch counts.  names[i] points to static strings. */
PPD_API int ppd_timing_enable(ppd_ctx *ctx, int32_t enable);
PPD_API int ppd_timing_collect(ppd_ctx *ctx);
PPD_API int ppd_timing_read(ppd_ctx *ctx, int32_t n, const char **names, double *ms, int64_t *launches,
                    int32_t *n_out);

/* Failure detection of the bounded device waits.  The degridding kernel waits
 * on an mbarrier for each TMA tile copy; the wait gives up after `polls`
 * polls (default PPD_WAIT_LIMIT_DEFAULT), sets the context's device error
 * word and, with the copies it started waited for under the default bound,
 * leaves the kernel; the next synchronising call (ppd_iterate with stats,
 * ppd_set_weights) returns PPD_ERR_TIMEOUT and clears the word, and the
 * context stays usable.  Setting a smaller limit (0: give up at once) makes
 * the first wait of every tile run out, which tests that path without any
 * fault; the results of the launches it affects are not defined.  Synchronises.
 * Errors: INVALID_ARG (NULL, polls < 0), CUDA. */
#define PPD_WAIT_LIMIT_DEFAULT (1ll << 21)
PPD_API int ppd_set_wait_limit(ppd_ctx *ctx, int64_t polls);

/* Kernel launches enqueued by this context since creation (all entry points). */
PPD_API int64_t ppd_launch_count(ppd_ctx *ctx);

/* Static description of a status code. */
PPD_API const char *ppd_status_string(int status);

/* Message of the calling thread's last failed call ("" if none). */
PPD_API const char *ppd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PPD_H */
