/*
 * mapmaker.h -- C ABI of the GB300 map-making library (libmapmaker.so).
 *
 * The library solves the map-making system of Puglisi et al., "Iterative
 * map-making with two-level preconditioning for polarized CMB data sets":
 *
 *   A x = b,   A = P^T W P,   b = P^T W d                 (Sect. 3, Eq. linearsystem)
 *
 * where P is the pointing matrix with rows (1, cos 2psi_t, sin 2psi_t) on the
 * pixel seen by sample t (Sect. 2, Eq. datamodel) and W = N^-1 is the
 * inverse-noise weight, here a symmetric banded Toeplitz matrix for each
 * stationary (detector, interval) block (any SPD weight gives an unbiased
 * estimate, Sect. 2, Eq. estimator).  PCG (Sect. 3, Eq. pcg) runs with the
 * block-diagonal preconditioner M_BD (Sect. 3.1, Eq. mbd) or the two-level
 * preconditioner M_2l = M_BD (1 - A Z E^-1 Z^T) + Z E^-1 Z^T, E = Z^T A Z
 * (Sect. 3.2, Eq. m2l), whose deflation basis Z holds Ritz vectors of
 * M_BD A from the Arnoldi process (Sect. 6; Appendix A, Algorithm arnoldi).
 *
 * Conventions shared by every call
 *  - Status codes only; no C++ exception crosses this boundary.  After a
 *    failure mm_last_error() returns a message owned by the context.
 *  - Maps at the boundary are float64 arrays [nrhs][n_pix][3] holding
 *    (I, Q, U) per pixel, whatever the precision of the context.
 *  - Timelines (TOD) at the boundary are [nrhs][n_samples] of float64 for an
 *    MM_FP64 context and of float32 for an MM_FP32_MIXED context.
 *  - Arguments tagged "mem" take MM_HOST (pageable or pinned host memory) or
 *    MM_DEVICE (device memory on the context's device).  The caller keeps
 *    ownership of every pointer it passes; the library copies what it keeps.
 *  - Work is ordered on the context's CUDA stream.  Calls return after the
 *    results they write to host memory (maps, info, counts) are complete;
 *    device outputs are complete once the stream reaches the call's end.
 *  - A context is not thread safe: one host thread at a time per context.
 *  - Every call makes the context's device current while it runs and gives
 *    the caller back the device that was current before.
 */
#ifndef MAPMAKER_H
#define MAPMAKER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_ctx mm_ctx;

typedef enum {
    MM_OK = 0,
    MM_ERR_ARG = 1,            /* invalid argument (message says which)          */
    MM_ERR_OOM = 2,            /* device allocation failed or budget exceeded     */
    MM_ERR_CUDA = 3,           /* a CUDA runtime call failed                      */
    MM_ERR_STATE = 4,          /* call out of order (e.g. solve before setup)     */
    MM_ERR_NOT_CONVERGED = 5,  /* PCG hit max_iter; the map is still written     */
    MM_ERR_BREAKDOWN = 6,      /* p^T A p <= 0 or a NaN appeared                  */
    MM_ERR_SINGULAR = 7,       /* coarse operator E is not SPD, or an eigen-solve */
                               /* of H_m / T_m did not converge                   */
    MM_ERR_TIMEOUT = 8,        /* reserved for a bounded device wait that gives   */
                               /* up; no kernel of this library waits on another  */
    MM_ERR_REDUCE = 9          /* the caller's cross-rank sum (mm_set_reduction)  */
                               /* reported a failure                              */
} mm_status;

typedef enum {
    MM_FP64 = 0,        /* gather, filter and scatter in float64                 */
    MM_FP32_MIXED = 1   /* gather/filter/scatter in float32 with float32
                           accumulation; PCG vectors, inner products, residual
                           norms, Arnoldi orthogonalisation, E and M_BD in
                           float64; the solve refines against a float64 A x   */
} mm_precision;

typedef enum { MM_PRECOND_BD = 0, MM_PRECOND_2L = 1 } mm_precond;

enum { MM_HOST = 0, MM_DEVICE = 1 };

typedef struct {
    int32_t iters;          /* products with A inside PCG                         */
    int32_t status;         /* mm_status of this right-hand side                  */
    double rel_res;         /* final recurrence residual ||r_k|| / ||b||          */
    double true_rel_res;    /* ||b - A x|| / ||b|| with a float64 product at exit  */
    double t_solve_ms;      /* device time of the whole solve call                */
    int32_t refinements;    /* outer float64 residual refinements (mixed mode)    */
    int32_t precond_used;   /* mm_precond applied to this right-hand side (M_BD   */
                            /* when "coarse_fallback" replaced M_2l, see options) */
} mm_solve_info;

/* Create a context on CUDA device `device`, ordered on `cuda_stream`
 * (a cudaStream_t; NULL means the legacy default stream).  *out receives the
 * context, which owns all device memory it allocates.  A process drives one
 * device (several contexts, on several host threads, may share it; use one
 * process per GPU for several GPUs): a context on another device than the
 * process's first one is refused with MM_ERR_ARG.  Errors: MM_ERR_ARG,
 * MM_ERR_CUDA. */
mm_status mm_create(mm_ctx** out, int device, void* cuda_stream, mm_precision prec);

/* Release the context and every device buffer it owns.  NULL is accepted. */
mm_status mm_destroy(mm_ctx* ctx);

/* Message of the last failure on this context ("" if none).  The pointer
 * stays valid until the next call on the context. */
const char* mm_last_error(const mm_ctx* ctx);

/* Pointing P and weight W (Sect. 2, Eq. datamodel and Eq. estimator).
 *  n_samples        timeline length N_t.
 *  n_det            the timeline is n_det equal detector timelines laid end to
 *                   end (n_samples % n_det == 0); per-RHS lengths in mm_solve
 *                   count samples per detector.  Use 1 for a single timeline.
 *  n_pix            pixels; unknowns are (I, Q, U) per pixel.
 *  pix [n_samples]  pixel of each sample, -1 marks a flagged sample (zero row
 *                   of P); values must lie in [-1, n_pix), checked
 *                   (MM_ERR_ARG) for host and device arrays alike.
 *  psi [n_samples]  HWP angle in radians; the row of P is (1, cos 2psi, sin 2psi).
 *  n_blocks, block_off [n_blocks+1]  stationary blocks [off_b, off_{b+1}),
 *                   contiguous, increasing, block_off[0] = 0,
 *                   block_off[n_blocks] = n_samples, none straddling two
 *                   detector timelines.
 *  block_band [n_blocks]  band index of each block, in [0, n_bands).
 *  half_bw          lambda >= 0; band [n_bands][half_bw+1] holds c_0..c_lambda
 *                   of each symmetric banded Toeplitz W block (host float64).
 *                   Within a block W_{tt'} = c_|t-t'| for |t-t'| <= lambda and
 *                   the band is cut at the block edges.  The caller guarantees
 *                   W is SPD.
 *  mem              where pix and psi live; block_off, block_band and band are
 *                   always host arrays.
 * Replaces any earlier pointing and drops M_BD and the coarse space.
 * Errors: MM_ERR_ARG (sizes, ranges), MM_ERR_OOM, MM_ERR_CUDA. */
mm_status mm_setup_pointing(mm_ctx* ctx, int64_t n_samples, int32_t n_det, int32_t n_pix,
                            const int32_t* pix, const float* psi,
                            int32_t n_blocks, const int64_t* block_off, const int32_t* block_band,
                            int32_t n_bands, int32_t half_bw, const double* band, int mem);

/* Block-diagonal preconditioner M_BD^-1 = P^T diag(W) P (Sect. 3.1, Eq. mbd):
 * one 3x3 block per pixel, summed and inverted in float64.  A pixel with fewer
 * than 3 hits or with lambda_min/lambda_max of its block below rcond_min is
 * dropped: its samples are flagged (pixel -1) in the context's copy of P, so
 * A and every later product exclude it, and its map entries solve to 0.
 * *n_dropped_out (may be NULL) receives the number of dropped pixels.
 * Errors: MM_ERR_STATE (no pointing), MM_ERR_ARG, MM_ERR_CUDA. */
mm_status mm_build_bd(mm_ctx* ctx, double rcond_min, int32_t* n_dropped_out);

/* b = P^T W d (Sect. 3, Eq. linearsystem) for nrhs timelines, computed to
 * float64 accuracy whatever the context precision (native float64, or
 * double-float arithmetic, see option "fp64_products").  tod [nrhs][n_samples] (element
 * type per context precision), b_out [nrhs][n_pix][3] float64, both in `mem`.
 * Errors: MM_ERR_STATE, MM_ERR_ARG, MM_ERR_OOM, MM_ERR_CUDA. */
mm_status mm_rhs(mm_ctx* ctx, const void* tod, double* b_out, int32_t nrhs, int mem);

/* y = A x = P^T W P x (Sect. 3, Eq. linearsystem), matrix-free, with the
 * operator the solver uses (float32 in MM_FP32_MIXED; in MM_FP64 native
 * float64 or double-float as option "fp64_products" says; option
 * "apply_precision" overrides): gather, banded-Toeplitz filter (or the
 * template filters) and scatter-add fused in one pass per sample segment.
 * x, y [nrhs][n_pix][3] float64 in `mem`.
 * Errors: MM_ERR_STATE, MM_ERR_ARG, MM_ERR_OOM, MM_ERR_CUDA. */
mm_status mm_apply_A(mm_ctx* ctx, const double* x, double* y, int32_t nrhs, int mem);

/* y = M x for M = M_BD (Sect. 3.1, Eq. mbd) or M_2l (Sect. 3.2, Eq. m2l).
 * x, y [nrhs][n_pix][3] float64 in `mem`.  Needs mm_build_bd, and for M_2l a
 * coarse space.  Errors: MM_ERR_STATE, MM_ERR_ARG, MM_ERR_CUDA. */
mm_status mm_apply_precond(mm_ctx* ctx, mm_precond which, const double* x, double* y,
                           int32_t nrhs, int mem);

/* Coarse space for M_2l (Sect. 6; Appendix A).  Runs Arnoldi on
 * B = M_BD A from r_0 = M_BD b (b [n_pix][3] float64 in `mem`; NULL uses the
 * first right-hand side of the last mm_rhs/mm_solve call), with two classical
 * Gram-Schmidt passes per step in float64, stopping when h_{j+1,j} <= eps_arn
 * or after m_max steps.  Ritz pairs of H_m (Eq. ritz) are sorted by real part;
 * the k smallest (or, if k <= 0, all with real part below eps_lambda, at most 512) form Z,
 * a complex pair adding its real and imaginary parts.  Z is orthonormalised,
 * AZ = A Z and E = Z^T A Z are formed, and E is factored (float64).
 * Ritz values at the round-off level of the largest (null directions of A)
 * are not used.  1 <= m_max <= 1024, k <= 512.
 * *k_out (may be NULL) receives dim Z.  Needs mm_build_bd.
 * Errors: MM_ERR_STATE, MM_ERR_ARG, MM_ERR_OOM, MM_ERR_SINGULAR, MM_ERR_CUDA. */
mm_status mm_build_coarse(mm_ctx* ctx, const double* b_or_null, int32_t m_max, double eps_arn,
                          int32_t k, double eps_lambda, int32_t* k_out, int mem);

/* Coarse space from the last M_BD solve instead of a separate Arnoldi run.
 * With option "harvest" = m > 0, a solve with M_BD keeps, for its first
 * right-hand side and first inner PCG run, the vectors v_j = z_j / sqrt(r_j^T z_j)
 * (z_j = M_BD r_j) and the coefficients alpha_j, beta_j for j < m.  PCG with
 * M_BD is the Lanczos process of B = M_BD A in the M_BD^-1 inner product, so
 * B V = V T_m + (rank one) with T_m tridiagonal, diagonal
 * 1/alpha_j + beta_{j-1}/alpha_{j-1} and off-diagonal -sqrt(beta_j)/alpha_j.
 * Ritz pairs of T_m (Appendix A, Eq. ritz, in its symmetric form) give the
 * deflation basis: the k smallest (or, if k <= 0, those below eps_lambda, at most 512)
 * form Z = V S, then Z is orthonormalised and AZ, E = Z^T A Z formed as in
 * mm_build_coarse (k <= 512).  *k_out (may be NULL) receives dim Z.
 * Errors: MM_ERR_STATE (no harvested solve), MM_ERR_ARG, MM_ERR_SINGULAR,
 * MM_ERR_CUDA. */
mm_status mm_build_coarse_from_solve(mm_ctx* ctx, int32_t k, double eps_lambda, int32_t* k_out);

/* Install a deflation basis Z [k][n_pix][3] float64 (`mem`) instead of
 * building one: the paper's "simplified" reuse of a basis computed on another
 * data subset (Sect. 7).  AZ and E = Z^T A Z are formed with this context's A;
 * 1 <= k <= 512.
 * Errors: MM_ERR_STATE, MM_ERR_ARG, MM_ERR_SINGULAR, MM_ERR_CUDA. */
mm_status mm_set_coarse(mm_ctx* ctx, int32_t k, const double* Z, int mem);

/* Copy out the current basis Z [k][n_pix][3] (host, may be NULL), the Ritz
 * values kept [k] (host, may be NULL) and k.  Errors: MM_ERR_STATE. */
mm_status mm_get_coarse(mm_ctx* ctx, double* Z_out, double* ritz_out, int32_t* k_out);

/* Checkpoint of the coarse space, for the paper's "simplified" reuse of one
 * scan's deflation basis across runs (Sect. 7) without recomputing A Z and E:
 * the basis Z, A Z, E^-1 (Sect. 3.2, Eq. m2l) and the Ritz values are written
 * to a host buffer with a 64-bit fingerprint of the operator they belong to
 * (pointing after pixel selection, weights, block structure, template
 * filters, product precision).
 * mm_export_coarse: buf NULL sets *bytes to the size needed; otherwise buf
 *   (host, *bytes long) receives the checkpoint and *bytes its size.
 *   Errors: MM_ERR_STATE (no coarse space), MM_ERR_ARG (buffer too small),
 *   MM_ERR_CUDA.
 * mm_import_coarse: installs a checkpoint (host buffer of `bytes`) into a
 *   context whose operator has the same fingerprint; needs mm_build_bd.  A
 *   checkpoint of another scan, filter or product precision, a truncated or
 *   foreign buffer, is refused with MM_ERR_ARG (use mm_set_coarse to reuse a
 *   basis on another scan: it forms A Z and E anew).  Errors: MM_ERR_STATE,
 *   MM_ERR_ARG, MM_ERR_OOM, MM_ERR_CUDA. */
mm_status mm_export_coarse(mm_ctx* ctx, void* buf, int64_t* bytes);
mm_status mm_import_coarse(mm_ctx* ctx, const void* buf, int64_t bytes);

/* Sum over ranks for a map-making problem whose timeline is split across
 * processes (one GPU each): A = P^T W P and b = P^T W d are sums over the
 * stationary blocks (Sect. 3, Eq. linearsystem), so a rank that sets up the
 * pointing of its own blocks (mm_setup_pointing with its samples only, the
 * same n_pix on every rank) forms partial products, and one element-wise sum
 * of each partial map over the ranks completes them; the PCG vectors, dot
 * products, M_BD and the coarse space are then replicated and every rank
 * follows the same iterations.  The library calls
 *     fn(buf, count, elem_bytes, user)
 * after every operator product (A x, b, the refinement residuals; 4 values
 * per pixel and right-hand side, the fourth 0) and on the M_BD sums (7 per
 * pixel); fn must replace buf by its sum over all ranks, in place, before it
 * returns, and return 0 (anything else fails the call with MM_ERR_REDUCE).
 * elem_bytes is 4 (float32 products) or 8 (float64).  on_device = 1 passes the
 * device buffer (for a device collective such as an NCCL all-reduce; the
 * context's stream is synchronised before the call); 0 stages it through a
 * host buffer (for a host collective such as gloo or MPI).  Every rank must
 * make the same sequence of calls.  fn = NULL switches the reduction off.
 * While a reduction is set, right-hand sides of uneven length, template
 * filters and captured CUDA graphs are refused (MM_ERR_ARG) or not used, and
 * automatic plan tuning runs without calling fn.
 * Errors: MM_ERR_ARG. */
typedef int (*mm_reduce_fn)(void* buf, int64_t count, int32_t elem_bytes, void* user);
mm_status mm_set_reduction(mm_ctx* ctx, mm_reduce_fn fn, void* user, int on_device);

/* Solve A x = b for nrhs timelines with PCG (Sect. 3, Eq. pcg), x_0 = 0,
 * stopping when ||r_k|| / ||b|| <= tol (recurrence residual) or after max_iter
 * products with A.  In MM_FP32_MIXED the float32 operator drives PCG and
 * float64 residuals b - A x refine the solution until the float64 residual
 * meets tol.
 *  tod [nrhs][n_samples] in `mem`; map_out [nrhs][n_pix][3] float64 in `mem`.
 *  rhs_len_or_null [nrhs] (host): samples per detector used by each
 *      right-hand side (its timelines are the first rhs_len[i] samples of each
 *      detector, as in a Monte Carlo batch of uneven lengths); each then has
 *      its own A_i and M_BD,i, while a coarse space, if any, is shared.  NULL
 *      uses whole timelines.
 *  info [nrhs] (host, may be NULL) receives per-RHS results.
 * Returns MM_OK when every right-hand side converged, MM_ERR_NOT_CONVERGED
 * when one did not (maps are written either way), MM_ERR_BREAKDOWN on a
 * non-positive p^T A p or a NaN.  Other errors: MM_ERR_STATE, MM_ERR_ARG,
 * MM_ERR_OOM, MM_ERR_CUDA. */
mm_status mm_solve(mm_ctx* ctx, const void* tod, double* map_out, int32_t nrhs,
                   const int64_t* rhs_len_or_null, mm_precond precond, double tol,
                   int32_t max_iter, mm_solve_info* info, int mem);

/* Tuning knobs, by name.  "filter": 0 auto, 1 direct band, 2 FFT;
 * "fft_len": FFT length 2^a 3^b (b <= 2) of the FFT filter, 0 = choose;
 * "fft_log2": FFT length 2^v (0 = choose); "autotune": 1 (default) times the
 * candidate filter plans on first use of a problem shape and keeps the
 * fastest (cached per process, and in the JSON-lines file named by the
 * environment variable MM_TUNE_CACHE when set); "direct_tile": outputs per
 * CTA of the direct filter; "check_every": PCG iterations between host
 * convergence checks; "graphs": 1 to replay a captured CUDA graph of
 * check_every PCG iterations (only on a created stream, not the legacy
 * default stream); "harvest": Lanczos vectors kept from M_BD solves (see
 * mm_build_coarse_from_solve); "time_filter": 1 records CUDA events around
 * every filter launch; "fp64_products": 1 native float64 or 2 (default for
 * MM_FP32_MIXED) double-float arithmetic (float32 pairs, about 44 bits) for
 * b and the refinement residuals, and in MM_FP64 for every operator product
 * as well (PCG, Arnoldi, A Z, mm_apply_A; vectors, dot products and the
 * coarse space stay float64); MM_ERR_STATE while a solve is in progress;
 * "apply_precision": precision of mm_apply_A (0 context, 1 float64,
 * 2 double-float); "inner_tol": in
 * MM_FP32_MIXED, the smallest relative tolerance asked of a float32-operator
 * PCG run between float64-accurate refinements (default 2e-6);
 * "half_transform": 1 (default) lets a whole block of N real samples run as
 * one N/2-point complex transform per CTA (paired real-spectrum step), 0
 * keeps two blocks per N-point transform; "coarse_prefix": 1 (default) forms
 * the per-RHS coarse products A_i Z of an uneven-length two-level batch from
 * products over whole blocks computed once per coarse space (block-diagonal
 * W; needs the same block boundaries in every detector) plus the one partly
 * covered block per detector, 0 forms every A_i Z directly;
 * "coarse_fallback": 1 (default) in a two-level batch of uneven length runs
 * M_BD for every right-hand side whose length differs by more than 1 % from
 * that of the operator the basis Z was built from (a prefix covers the patch
 * differently and its small eigenmodes are not in span Z: M_2l would cost
 * more for the same products), and M_BD for the whole batch when none is
 * left; info[i].precond_used says which ran; 0 keeps M_2l for all;
 * "tc_coarse": 1 (default) forms the coarse products Z^T R, Z U and A Z U of
 * M_2l (Sect. 3.2, Eq. m2l) on the tensor cores (tcgen05, TF32 operands split
 * in high and low parts, about 21 bits) when 8 <= nrhs <= 128, k <= 64, the
 * right-hand sides share one coarse space and the map has at least 16384
 * pixels (smaller maps are faster in float64 on the CUDA cores); 2 does so
 * for every eligible batch whatever the map size; 0 keeps them in float64.  A bounded wait of the tensor-core kernels that gives up is
 * reported as MM_ERR_TIMEOUT.  Errors: MM_ERR_ARG for an unknown name or
 * value. */
mm_status mm_set_option(mm_ctx* ctx, const char* name, double value);

/* Read back a tuning knob or statistic: any knob above, or "last_apply_ms"
 * (device time of the last mm_apply_A), "filter_launches" and "filter_ms"
 * (filter launches timed since the last read of "filter_ms", and their total
 * device time; reading "filter_ms" resets both), "kernel_launches" (kernels
 * launched by the library since load), "plan_fft_len", "plan_fft_log2",
 * "plan_whole" (the plan a single-RHS product uses: 0 overlap-save segments,
 * 1 whole blocks two per transform, 2 whole blocks as half-length complex
 * transforms), "harvested" (Lanczos
 * vectors kept by the last M_BD solve), "device_bytes" (device memory in use),
 * "coarse_len" (samples per detector of the operator the basis was built from),
 * "coarse_rank_min" (the fewest coarse vectors a right-hand side of the last
 * uneven two-level batch kept: a prefix of the scan that leaves part of the map
 * unobserved makes E_i = Z^T A_i Z semi-definite, and M_2l,i then uses the
 * columns of Z that a pivoted Cholesky factorisation of E_i keeps).
 * Errors: MM_ERR_ARG, MM_ERR_STATE. */
mm_status mm_get_option(mm_ctx* ctx, const char* name, double* value);

/* Stepwise solve for schedulers that interleave many solves (continuous
 * batching).  mm_solve_begin sets up the same solve as mm_solve and runs no
 * iteration; mm_solve_step runs up to n_iter PCG iterations (enqueued on the
 * context stream) and sets *done to 1 once every right-hand side has
 * converged or reached max_iter; mm_solve_end writes maps and info exactly
 * like mm_solve and returns its status.  Steps of different contexts on
 * different streams overlap on the device. */
mm_status mm_solve_begin(mm_ctx* ctx, const void* tod, int32_t nrhs, const int64_t* rhs_len_or_null,
                         mm_precond precond, double tol, int32_t max_iter, int mem);
mm_status mm_solve_step(mm_ctx* ctx, int32_t n_iter, int32_t* done);
mm_status mm_solve_end(mm_ctx* ctx, double* map_out, mm_solve_info* info, int mem);

/* Non-blocking stepping for a scheduler that drives many contexts from one
 * host thread.  mm_solve_launch enqueues n_iter PCG iterations and an
 * asynchronous read-back of the per-RHS state and returns at once;
 * mm_solve_poll sets *ready to 1 once that read-back has landed (0 while the
 * device is still busy) and then *done as mm_solve_step would; a finished
 * inner solve may start a float64 refinement before returning.  Errors:
 * MM_ERR_STATE (no solve begun, or poll without launch), MM_ERR_ARG,
 * MM_ERR_CUDA. */
mm_status mm_solve_launch(mm_ctx* ctx, int32_t n_iter);
mm_status mm_solve_poll(mm_ctx* ctx, int32_t* ready, int32_t* done);

/* Template filters of ground-based scans (Sect. 2.1, Eq. filt, Eq.
 * filtnoise, Eq. unb; Sect. 4; Sect. 5.1).  After this call the context's
 * operator is A = P^T F P and b = P^T F d with the symmetric simplified filter
 * F = F_B W^-1 F_G W^-1 F_B, F_X = W - W X (X^T W X)^-1 X^T W, W = w_b I on
 * block b (w_b = c_0 of the block's band: the pointing must have been set up
 * with half_bw = 0, white weights).
 *  poly_order      K in -1..3: X = B holds the Legendre polynomials P_0..P_K
 *                  of u = 2 (i + 1/2)/m - 1 over each subscan of m samples
 *                  (order min(K, m - 1) on subscans of m <= K samples);
 *                  -1: no polynomial filter.
 *  subscan_off     [n_subscans + 1] HOST array of sample offsets, 0 ..
 *                  n_samples, strictly increasing, every subscan inside one
 *                  block (block boundaries are subscan boundaries).  May be
 *                  NULL when poly_order < 0.
 *  az_bin          [n_samples] azimuth bin of every sample (-1: none), host
 *                  or device per `mem`; X = G holds one indicator column per
 *                  bin and per block (a block is one constant-elevation
 *                  scan).  NULL: no ground filter.  1 <= n_az_bins <= 8192.
 *  stokes          0: pointing rows (1, cos 2psi, sin 2psi) (I, Q, U);
 *                  1: rows (0, cos 2psi, sin 2psi) -- the differenced
 *                  timeline d^- of Sect. 5.1 (Eq. d-); I is not solved for
 *                  (M_BD inverts the 2x2 (Q, U) block, a pixel needs 2 hits
 *                  and rcond >= rcond_min of that block);
 *                  2: rows (1, 0, 0) -- the summed timeline d^+ (Eq. d+,
 *                  intensity maps of App. B); Q, U are not solved for (1x1
 *                  M_BD, 1 hit).  With polynomial templates a constant I map
 *                  is then an exact null vector of A: the solve converges in
 *                  the range of A and leaves that component at 0.
 * The filters act on every sample, flagged ones included.  Calling with
 * poly_order = -1, az_bin = NULL and stokes = 0 restores the band weight.
 * Clears M_BD and the coarse space (rebuild them) and sets "fp64_products"
 * to 1 (native float64); set it to 2 afterwards for double-float products.
 * Right-hand sides of uneven length (rhs_len) are not supported with
 * templates (MM_ERR_ARG at solve time).  The longest block and the bins must
 * fit shared memory: 8 bytes per sample + 12 bytes per bin <= 220 KB.
 * Errors: MM_ERR_ARG, MM_ERR_STATE (no pointing), MM_ERR_OOM, MM_ERR_CUDA. */
mm_status mm_set_templates(mm_ctx* ctx, int32_t poly_order, int32_t n_subscans, const int64_t* subscan_off,
                           const int32_t* az_bin, int32_t n_az_bins, int32_t stokes, int mem);

/* M_2l applied without allocating device memory during the call (the paper
 * has no counterpart; this is a deployment variant of mm_apply_precond).
 * For callers that must not call cudaMalloc/cudaFree while they run: latency-
 * critical serving loops (allocation can synchronise the device and can fail
 * under memory pressure) and host applications or plug-ins whose device
 * memory belongs to another allocator.
 *  x, y   [nrhs][n_pix][3] float64, DEVICE memory on the context's device,
 *         owned by the caller; y = M_2l x as mm_apply_precond computes it.
 *         x and y must not overlap (MM_ERR_ARG): the call does not work in
 *         place.
 *  Needs mm_build_bd and a coarse space (those calls allocate; this one
 *  does not).  Reduction scratch lives in a fixed 1 MiB device array inside
 *  the library, held by every GPU that loads it until the process exits.
 *  Limits: nrhs <= 128, k <= 128 and 2 * nrhs * k + 64 <= 131072; larger
 *  requests return MM_ERR_ARG.  The first call on a device looks up the
 *  array's device address (cudaGetSymbolAddress); make that first call
 *  before any stream capture.  All calls share the array, so calls that
 *  overlap on the GPU (other streams or threads) race; serialise them.
 *  The call blocks until the result is complete (it synchronises the
 *  context's stream) and leaves the caller's current device as it found it.
 *  The looked-up address lasts for the life of the process; like the
 *  contexts, it does not survive a cudaDeviceReset.  Errors: MM_ERR_ARG,
 *  MM_ERR_STATE, MM_ERR_CUDA. */
mm_status mm_apply_precond_2l_noalloc(mm_ctx* ctx, const double* x, double* y, int32_t nrhs);

/* Device bytes a context needs for a problem of this shape (pointing, maps,
 * PCG state, Arnoldi basis of m_max vectors and k coarse vectors), for
 * admission control, with the default options ("fp64_products" = 2 in
 * MM_FP64 adds 16 bytes per sample of double-float weights).  Pure host
 * arithmetic; needs no device. */
int64_t mm_estimate_bytes(int64_t n_samples, int32_t n_pix, int32_t n_bands, int32_t half_bw,
                          int32_t nrhs, int32_t m_max, int32_t k, mm_precision prec);

/* Measured FMA rate of the CUDA cores of `device` (not a step of the paper's
 * method: the denominator of the arithmetic view of the filter kernels'
 * roofline).  fp64 = 0 times float32 FMAs, 1 float64; the timed launch runs
 * for about `seconds` (0 < seconds <= 60) on every SM (8 independent FMA
 * chains per thread, 2048 threads per SM).  *flops_per_s receives 2 flop per
 * FMA per second.  It allocates a small device buffer and leaves the caller's
 * current device as it found it.  Errors: MM_ERR_ARG, MM_ERR_OOM, MM_ERR_CUDA. */
mm_status mm_fma_peak(int device, int fp64, double seconds, double* flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* MAPMAKER_H */
