/*
 * lcmg.h -- C ABI of liblcmg.so: multigrid-preconditioned CG for the
 * regularized least-squares problems of Bolten, MacLachlan and Kilmer,
 * "Multigrid preconditioning for regularized least-squares problems".
 *
 * The library solves, for a list of regularization parameters lambda_i and
 * right-hand sides b, the regularized normal equations
 *
 *     (A^T A + lambda^2 L^T D^2 L) x = A^T b                 (Sec. 3.2, eq. (normal))
 *
 * where A is the forward operator (a CSR matrix, e.g. a CT ray-length
 * matrix, or a blur PSF applied with zero boundary), L the discrete gradient
 * of an n_v x n_h image (Sec. 2, eq. (gradient)) and D = diag(d) the edge
 * weights of the outer iteration (Sec. 2, eq. (g)).  Each system is solved
 * by preconditioned CG; the preconditioner is one symmetric multigrid
 * V-cycle (Algorithm 1) on lambda^2 L^T D^2 L + diag(A^T A) with Galerkin
 * coarse operators (Sec. 3.1).  The outer loop of Algorithm 2 (L-curve
 * corner, weight update, lambda trimming, stopping rule) is exposed both
 * as separate calls and end to end.
 *
 * Conventions
 *  - Images are n_v x n_h, vectorised column-major: pixel (i, j) -> i + j*n_v.
 *  - Edge vectors (d, D L x) hold the n_h*(n_v-1) vertical differences
 *    first, then the (n_h-1)*n_v horizontal ones, each column-major (the
 *    row order of L in eq. (gradient)).
 *  - Lambda lists are strictly increasing (Sec. 3.4 indexes them that way);
 *    index arguments are 1-based like the paper's i.
 *  - Every call returns an lcmg_status; nothing throws across the ABI.
 *    lcmg_last_error() returns a message for the calling thread's most
 *    recent failure.
 *  - Ownership: the caller owns every buffer it passes.  Host-pointer calls
 *    copy inputs into device memory the context owns (freed by
 *    lcmg_destroy) and copy results back before returning.  *_dev calls
 *    take device pointers valid on the context's device, read and write them
 *    in stream order on the context's stream, never free them, and return
 *    without synchronising unless stated.
 *  - Device pointers and streams are passed as void* (a cudaStream_t).
 *  - A context is not thread safe; use one per host thread.
 */
#ifndef LCMG_H
#define LCMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------- */
typedef enum {
  LCMG_OK = 0,
  LCMG_ERR_INVALID_ARG = 1,  /* bad size, pointer, order, or inconsistent state  */
  LCMG_ERR_NOMEM = 2,        /* device allocation failed or over the HBM budget  */
  LCMG_ERR_CUDA = 3,         /* a CUDA runtime call failed                        */
  LCMG_ERR_NOT_READY = 4,    /* server: result not available yet                 */
  LCMG_ERR_CANCELLED = 5,    /* server: request cancelled or timed out            */
  LCMG_ERR_STATE = 6         /* call made before the state it needs was set       */
} lcmg_status;

/* per-system outcome written to status[] by the solve calls */
typedef enum {
  LCMG_CONVERGED = 0,        /* ||A^T b - K x||_2 <= tol ||A^T b||_2 (true residual) */
  LCMG_MAXIT = 1,            /* iteration limit reached                              */
  LCMG_BREAKDOWN = 2,        /* p^T K p <= 0 or r^T z <= 0                           */
  LCMG_NONFINITE = 3         /* NaN or Inf met                                       */
} lcmg_solve_status;

typedef enum { LCMG_SMOOTH_L1_JACOBI = 0, LCMG_SMOOTH_JACOBI = 1 } lcmg_smoother;
typedef enum {
  LCMG_PREC_FP64 = 0,        /* all vectors, operators and reductions in FP64       */
  LCMG_PREC_MIXED = 1        /* FP32 SpMV/stencils/V-cycle, FP64 dots, alpha/beta,
                                true residuals (reliable updates) and coarse solve  */
} lcmg_precision;
typedef enum {
  LCMG_MODE_BATCHED = 0,     /* all (lambda, rhs) columns advanced together          */
  LCMG_MODE_SEQUENTIAL = 1   /* one lambda at a time, largest first, each warm-started
                                from the previous lambda's solution (Sec. 3.3)        */
} lcmg_mode;

/* ---- parameters ------------------------------------------------------ */
typedef struct {
  int32_t levels;       /* multigrid levels incl. the finest; 0 = coarsen by 2 while
                           both sides are even and one exceeds coarse_max            */
  int32_t coarse_max;   /* side limit of the coarsest grid for levels = 0 (default 16) */
  int32_t nu;           /* pre- = post-smoothing sweeps (default 1; equal counts keep
                           the V-cycle symmetric so CG applies; on the 256^2 CT
                           chain V(1,1) needs fewer PCG iterations than V(2,2)
                           and each is cheaper)                                     */
  int32_t smoother;     /* lcmg_smoother (default l1-Jacobi)                         */
  double omega;         /* damping of LCMG_SMOOTH_JACOBI (default 2/3)               */
  double q;             /* exponent of eq. (g) (default 2)                           */
  double d_min;         /* lower clamp of d in eq. (g) (default 1e-3)                */
  double tol;           /* relative normal-equations residual (default 1e-6)         */
  int32_t maxit;        /* PCG iteration limit per system (default 10000)            */
  int32_t precision;    /* lcmg_precision (default FP64)                             */
  int32_t mode;         /* lcmg_mode (default sequential: the paper's chain)          */
  int32_t check_every;  /* device iterations between host convergence polls (16)     */
  int32_t graphs;       /* 1 = replay each block of check_every iterations as one CUDA
                           graph (default), 0 = launch kernels one by one            */
  int32_t timing;       /* 1 = time the operator passes with CUDA events (see
                           lcmg_stats); default 0                                     */
  int32_t vfuse;        /* run each V-cycle level (nu = 1 or 2) as two kernels on
                           8 x 8 coarse-point tiles held in shared memory: pre-
                           smoothing + residual + restriction, then prolongation +
                           post-smoothing.  1 = for batches of at most 4 columns
                           (default), 2 = always, 0 = one kernel per step        */
  int32_t keep_direction; /* a column whose recursive residual met tol but whose
                           FP64 true residual did not: 1 = replace the residual
                           and continue from the current search direction
                           (residual replacement); 0 = restart with p = z
                           (default)                                            */
  int32_t autotune;     /* 1 = on the first solve of each batch width, time the
                           one-column SpMV configurations of the two operator
                           passes and both V-cycle forms on this context's
                           operator and keep the fastest (results may then
                           differ from an untuned context in the last bits:
                           the sums are taken in another order); 0 = fixed
                           defaults (default)                                   */
  int32_t spmv_variant; /* one-column SpMV configuration of both operator passes
                           (unless autotuned): 0 = per-pass default (32 lanes x
                           4 nonzeros for A p, 8 x 8 for the transposed pass,
                           as variant 4 with FP32 vectors);
                           1 = 32 x 4, 2 = 16 x 8, 3 = 8 x 8; with FP32 vectors
                           also 4 = 8 x 8 compiled for 5 resident blocks per SM
                           (48 registers), 5 = 8 x 8 for 6 blocks, 6 = 8 lanes
                           x 4 for 8 blocks (as 3 with FP64 vectors)           */
  int32_t stop_rule;    /* outer loop of Algorithm 2: 0 = stop after three equal
                           selections (Sec. 3.5, default); 1 = stop once
                           ||L x*||_2 decreases from one outer iteration to the
                           next (the heuristic of Gazzola et al. that Sec. 3.5
                           compares against); x_out is then the last selection */
  int32_t precond;      /* 0 = PCG with the V-cycle on lam^2 L^T D^2 L + diag(A^T A)
                           (default); 1 = the paper's own method (Sec. 3.2-3.3):
                           FGMRES preconditioned by a V(2,1) cycle on the whole
                           normal operator with one-sided coarse operators
                           A_{k+1} = A_k P_k, Jacobi-preconditioned CG relaxation
                           and an exact coarsest solve; CSR forward operators,
                           FP64 (precision = FP64; INVALID_ARG otherwise), one
                           lambda at a time (lcmg_apply_vcycle_dev then
                           applies this cycle)                              */
  int32_t gmres_restart; /* FGMRES basis size before a restart (1..2000; 200)     */
  int32_t coarsening;   /* interpolation of the paper's method (precond = 1):
                           0 = geometric cell-centred bilinear P on the grid
                           (default); 1 = classical AMG of Sec. 3.1 on
                           L^T D^2 L (strength theta = 0.25, the two-pass C/F
                           split, the paper's interpolation formula), rebuilt
                           on the host for every weight vector; 2 = the same
                           with the split by PMIS on the device
                           (lcmg_pmis_split) instead of the two passes;
                           `levels` is then the largest level count (0 = no
                           limit)                                           */
  int32_t amg_coarse_max; /* classical AMG: coarsen while a level has more
                           points than this (2..2048; 256); the last level is
                           solved densely                                   */
  int32_t compact_cols; /* one-column transposed pass (8-lane layout): 1 = read
                           column indices as 16-bit offsets from a per-row base
                           (6 instead of 8 bytes per FP32 nonzero; built by
                           set_forward_csr when every row of A and A^T spans
                           fewer than 65,536 columns, else int32 indices are
                           read; default); 0 = always int32.  Results are
                           bitwise identical                                 */
  int32_t alpha_fuse;   /* one column (batch of 1): 1 = every block of the x/r
                           update sums the p.q partials itself (fixed order)
                           and applies alpha = r.z / p.q, so no scalar kernel
                           runs between the operator and the update (default);
                           0 = a scalar kernel computes alpha first.  The two
                           sum in different orders (last-bit differences)  */
  int32_t beta_fuse;    /* one column with alpha_fuse and keep_direction = 0:
                           1 = every block of the p update sums the r.r and
                           r.z partials itself, takes the convergence /
                           limit / breakdown decision and applies
                           beta = r.z_new / r.z (default); 0 = a scalar kernel
                           computes beta first                             */
  int32_t spmv_variant_at; /* configuration of the transposed pass alone (0 =
                           as spmv_variant; 1..6 as there)                  */
  int32_t max_blocks;   /* cap on the blocks of every grid-stride launch (0 =
                           the default, 8 per SM up to 2048).  A small cap
                           makes each block, and each warp of the one-column
                           SpMV, walk many rows: the same sums in the same
                           order per row, for testing those loops           */
  int32_t smoother_fp16; /* mixed precision, a batch whose columns share one
                           lambda (the chain; its right-hand-side batches) and
                           the two-kernels-per-level cycle: 1 = the V-cycle's
                           smoother data in FP16 with power-of-two scales (the
                           finest level's edge weights and diag(A^T A); per
                           lambda the 24 off-diagonal coefficients of each
                           coarse K_k(lambda), with the diagonal rebuilt from
                           the FP32 row sums of G_A^k) (default); 0 = FP32.
                           The cycle stays symmetric positive definite; it
                           differs from the FP32 cycle by the rounding of its
                           coefficients to 11 bits                        */
} lcmg_params;

typedef struct lcmg_ctx lcmg_ctx;

/* Fill *p with the defaults listed above. */
void lcmg_default_params(lcmg_params* p);

/* Message of the calling thread's last failure ("" if none).  The string is
 * owned by the library and valid until the thread's next lcmg call. */
const char* lcmg_last_error(void);

/* Library version string. */
const char* lcmg_version(void);

/* Create a context on CUDA device `device` that launches on `stream` (a
 * cudaStream_t).  With stream = NULL the context creates a non-blocking
 * stream of its own (capturable into CUDA graphs, and not synchronised with
 * the legacy default stream, so contexts driven from several host threads
 * never join each other's captures).  Every copy the library makes runs on
 * the context's stream.  p may be NULL (defaults).
 * Errors: INVALID_ARG (bad device or parameters), CUDA. */
int lcmg_create(lcmg_ctx** ctx, int device, void* stream, const lcmg_params* p);

/* Free every device buffer the context owns.  Accepts NULL. */
int lcmg_destroy(lcmg_ctx* ctx);

/* Replace the parameters (takes effect at the next set_weights / solve). */
int lcmg_set_params(lcmg_ctx* ctx, const lcmg_params* p);

/* Define the image grid n_v x n_h and hence L (Sec. 2, eq. (gradient));
 * number of edges = n_h (n_v - 1) + (n_h - 1) n_v.  Resets weights to
 * D = I.  Errors: INVALID_ARG if n_v < 2 or n_h < 2. */
int lcmg_set_grid(lcmg_ctx* ctx, int32_t n_v, int32_t n_h);

/* Forward operator A as an m x n CSR matrix (n = n_v n_h) from host arrays:
 * row_ptr[m+1] (int64, row_ptr[0] = 0, non-decreasing), col[nnz] (int32,
 * 0 <= col < n), val[nnz] of dtype 0 = FP32 or 1 = FP64.  The library
 * copies them, builds A^T as a second CSR (no atomics at apply time) and
 * diag(A^T A) as column sums of squares (Sec. 3.2).  Requires set_grid.
 * Errors: INVALID_ARG (sizes, monotonicity, column range), STATE, NOMEM. */
int lcmg_set_forward_csr(lcmg_ctx* ctx, int64_t m, int64_t n, const int64_t* row_ptr,
                         const int32_t* col, const void* val, int32_t val_dtype);

/* Forward operator A as a kh x kw point-spread function (row-major, kh and
 * kw odd) applied as a zero-boundary correlation:
 *   (A x)(i, j) = sum_{u,v} psf[(u + kh/2) * kw + (v + kw/2)] x(i + u, j + v)
 * over pixels inside the image (rows of A truncated at the boundary, not
 * renormalised).  A^T uses the flipped PSF.  Requires set_grid. */
int lcmg_set_forward_stencil(lcmg_ctx* ctx, int32_t kh, int32_t kw, const double* psf);
/* A PSF that is an outer product fv fh^T (every entry within 1e-14 of the
 * largest of fv[u] fh[v], with fv the row sums and fh the column sums over
 * their total) is applied in its separable form, the Kronecker product of
 * two 1-D zero-boundary Toeplitz correlations (the deblurring example of
 * Sec. 4 builds its blur this way): A^T A = (A_h^T A_h) (x) (A_v^T A_v) as
 * two banded passes of 4r + 1 taps, A and A^T as passes of 2r + 1 taps.  The
 * result equals the 2-D form up to rounding.  Radii up to 16 (kh, kw <= 33);
 * larger PSFs use the 2-D form.  Errors: INVALID_ARG (even or zero sides,
 * PSF larger than 2 n + 1, non-finite values), STATE (no grid). */

/* Forward operator A given by its 1-D factors: the PSF fv fh^T with fv
 * (kh values, along i, the image columns) and fh (kw values, along j):
 *   (A x)(i, j) = sum_{u,v} fv[u + kh/2] fh[v + kw/2] x(i + u, j + v)
 * with zero boundary, i.e. A = A_h (x) A_v (Sec. 4, the Kronecker form of
 * the blur).  Uses the separable passes above (kh, kw <= 33), else the 2-D
 * form of the same PSF.  Requires set_grid; the library copies fv, fh.
 * Errors as lcmg_set_forward_stencil. */
int lcmg_set_forward_separable(lcmg_ctx* ctx, int32_t kh, const double* fv, int32_t kw,
                               const double* fh);

/* How the forward operator is applied: 0 none, 1 CSR, 2 PSF in its 2-D
 * form, 3 PSF in its separable form. */
int lcmg_forward_form(lcmg_ctx* ctx, int32_t* form);

/* Edge weights d of D = diag(d) (host array of n_edges values in (0, 1]).
 * Rebuilds the lambda-independent multigrid hierarchy on the device
 * (G_L^{k+1} = P^T G_L^k P, G_A^{k+1} = P^T G_A^k P, Sec. 3.1-3.2).
 * Errors: INVALID_ARG (count, non-positive or non-finite entries), STATE. */
int lcmg_set_weights(lcmg_ctx* ctx, const double* d, int64_t n_edges);
int lcmg_set_weights_dev(lcmg_ctx* ctx, const double* d_dev, int64_t n_edges);

/* Copy the current weights d (n_edges doubles) to a host buffer. */
int lcmg_get_weights(lcmg_ctx* ctx, double* d_out, int64_t n_edges);

/* Solve eq. (normal) for every (lambda_i, b_r) pair.
 *   lambda[n_lambda]    strictly increasing, > 0 (host)
 *   b[n_rhs][m]         right-hand sides, each contiguous (host)
 *   x0                  NULL (zero initial guesses) or [n_rhs][n_lambda][n]
 *   x[n_rhs][n_lambda][n]         solutions (host, written)
 *   resid_norm[n_rhs][n_lambda]   rho = ||A x - b||_2        (may be NULL)
 *   seminorm[n_rhs][n_lambda]     eta = ||D L x||_2          (may be NULL)
 *   iters, status [n_rhs][n_lambda]  PCG iterations and lcmg_solve_status
 *                                    (may be NULL)
 * Synchronises the stream before returning.  A system that does not
 * converge is reported in status[], not as an error. */
int lcmg_solve(lcmg_ctx* ctx, int32_t n_lambda, const double* lambda, int32_t n_rhs,
               const double* b, const double* x0, double* x, double* resid_norm,
               double* seminorm, int32_t* iters, int32_t* status);

/* As lcmg_solve with device pointers (same layouts; lambda stays on the
 * host).  x0_dev may equal x_dev (in-place warm start).  Returns once the
 * work is enqueued and the iteration has finished (the convergence poll
 * synchronises on the context's stream). */
int lcmg_solve_dev(lcmg_ctx* ctx, int32_t n_lambda, const double* lambda, int32_t n_rhs,
                   const double* b_dev, const double* x0_dev, double* x_dev,
                   double* resid_norm_dev, double* seminorm_dev, int32_t* iters_dev,
                   int32_t* status_dev);

/* L-curve corner (Sec. 1): index (0-based) of the point of maximum positive
 * signed Menger curvature of (log10 rho_i, log10 eta_i), i = 0..k-1 in
 * order of increasing lambda; ties within 1e-12 relative go to the smaller
 * lambda; with no positive curvature the maximum over interior points;
 * endpoints never.  Host only.  Errors: INVALID_ARG if k < 3 or a value is
 * not positive and finite. */
int lcmg_lcurve_corner(int32_t k, const double* rho, const double* eta, int32_t* idx);

/* Weight update of eq. (g) from x_star (n values, host): v = D L x_star,
 * g = |v| / ||v||_inf, d = max(1 - g^q, d_min), D <- diag(d) D; D unchanged
 * if v = 0.  Rebuilds the hierarchy.  d_out (n_edges, host) may be NULL. */
int lcmg_update_weights(lcmg_ctx* ctx, const double* x_star, double q, double d_min,
                        double* d_out);
int lcmg_update_weights_dev(lcmg_ctx* ctx, const double* x_star_dev, double q,
                            double d_min);

/* Classical AMG coarsening (Sec. 3.1) of an n x n matrix K in host memory
 * (CSR: row_ptr[n+1], column indices sorted within each row, FP64 values);
 * no device use.  j != i is a strong connection of row i when
 * -k_ij > theta * max_{m != i}(-k_im) * (1 + 1e-10) (a tie is weak; the paper
 * takes theta = 0.25).  First pass: greedy, largest number of strongly
 * dependent points first (ties: smallest index); a new C point's unsorted
 * dependants become F; each unsorted strong connection of a new F point gains
 * one.  Second pass, F points in increasing order: a strong F connection j of
 * i without a strong connection into i's strong C points C_i becomes C
 * tentatively (and joins C_i); a second such j makes i itself C instead.
 * cf[i] (n, caller-owned) = 1 for a C point, 0 for an F point.
 * Errors: INVALID_ARG for n < 1, a null pointer, a column out of range or
 * rows not sorted. */
int lcmg_rs_split(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                  double theta, int8_t* cf);

/* Interpolation of the split cf (as lcmg_rs_split returns, same K and
 * theta) by the formula of Sec. 3.1:
 *   w_ij = -(k_ij + sum_{m in F_i^s} k_im k_mj / sum_{l in C_i} k_ml)
 *          / (k_ii + sum_{m in F_i^w} k_im)
 * for the strong C connections j of an F point i (F_i^s its strong F
 * connections, F_i^w its other neighbours; a strong F connection whose sum
 * over C_i is zero counts with F_i^w); a C point injects.  Coarse points are
 * numbered in increasing fine index.  Output: P as CSR (p_row_ptr[n+1],
 * p_col / p_val with room for `cap` entries, caller-owned); *nnz = the
 * number of entries.  Errors: INVALID_ARG as lcmg_rs_split, or cap < *nnz
 * (then only *nnz is written). */
int lcmg_rs_interp(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                   double theta, const int8_t* cf, int64_t cap, int64_t* p_row_ptr,
                   int32_t* p_col, double* p_val, int64_t* nnz);

/* PMIS C/F split (De Sterck, Yang and Heys 2006), the parallel replacement
 * of lcmg_rs_split's two passes, run on the current CUDA device for a matrix
 * in host memory (same arguments and strength rule as lcmg_rs_split).
 * Measure of point i: |S_i^T| + u_i, u_i = (z >> 11) 2^-53 for the i-th
 * output z of the SplitMix64 stream seeded with `seed` (level k of a
 * context's hierarchy uses seed 2306 + k).  A point with no strong
 * connection in either direction is F; then, in rounds, every unsorted
 * point whose (measure, index) exceeds that of each unsorted point it is
 * strongly connected to (either direction) becomes C, and every unsorted
 * point with a strong connection to a C point becomes F.  cf[i] = 1 for C,
 * 0 for F.  Errors: as lcmg_rs_split; NOMEM or CUDA from the device. */
int lcmg_pmis_split(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                    double theta, uint64_t seed, int8_t* cf);

/* Level sizes of the classical AMG hierarchy the context last built
 * (coarsening = 1, after a solve): sizes[k] for k < min(cap, levels),
 * *n_levels = the level count.  Errors: STATE if none was built. */
int lcmg_amg_levels(lcmg_ctx* ctx, int32_t cap, int64_t* sizes, int32_t* n_levels);

/* Lambda window of Algorithm 2 (1-based, inclusive): i_prev = 0 marks the
 * first outer iteration (window 1..m); otherwise
 * [max(min(i_prev-2, m-9), 1), min(max(i_prev+7, 10), m)].  Host only. */
int lcmg_cull_lambdas(int32_t m, int32_t i_prev, int32_t* lo, int32_t* hi);

/* Algorithm 2 end to end for one right-hand side b[m] (host) and m_lambda
 * increasing lambdas: D^(1) = I; per outer iteration: window, hierarchy,
 * solves (warm-started from the previous outer iteration's solutions; zero
 * at the first), L-curve corner, stop after three equal selections or
 * max_outer iterations, else weight update.
 *   x_out[n]                 the final selected solution x^(i_l, l)
 *   lambda_idx_history[max_outer]  selected 1-based indices per iteration
 *   n_outer                  outer iterations run
 *   n_solves (may be NULL)   systems solved in total (sum of window sizes)
 *   n_converged (may be NULL) of which reached the tolerance */
int lcmg_lcurve_run(lcmg_ctx* ctx, int32_t m_lambda, const double* lambda, const double* b,
                    int32_t max_outer, double* x_out, int32_t* lambda_idx_history,
                    int32_t* n_outer, int64_t* n_solves, int64_t* n_converged);

/* Same with b and x_out as device pointers. */
int lcmg_lcurve_run_dev(lcmg_ctx* ctx, int32_t m_lambda, const double* lambda,
                        const double* b_dev, int32_t max_outer, double* x_out_dev,
                        int32_t* lambda_idx_history, int32_t* n_outer, int64_t* n_solves,
                        int64_t* n_converged);

/* Statistics of the last top-level call (solve or lcurve_run): total PCG
 * iterations over all systems, batched iterations issued, kernels launched,
 * and the milliseconds spent in the device iteration (CUDA events).  With
 * params.timing = 1 the two passes of every operator application
 * q = K p inside the PCG iteration (A p, then A^T y + lam^2 L^T W L p) are
 * bracketed by CUDA events on the context's stream: op_ms_a / op_ms_at
 * are their summed durations, op_launches the number of timed passes and
 * op_bytes their summed algorithmic (compulsory) DRAM bytes; the V-cycle
 * of the same iterations is bracketed too: vcycle_ms, vcycle_count and
 * vcycle_bytes (every level's vectors read and written once and its
 * smoother data read once per visit, as stored). */
typedef struct {
  int64_t column_iterations;
  int64_t batch_iterations;
  int64_t kernel_launches;
  double iterate_ms;
  double op_ms_a;
  double op_ms_at;
  int64_t op_launches;
  int64_t op_bytes;
  int32_t tuned_spmv_a, tuned_spmv_at;  /* SpMV configuration of the passes
                           (params.spmv_variant numbering: 1 = 32 lanes x 4,
                           2 = 16 x 8, 3 = 8 x 8, 4-6 the register-bounded
                           forms; 0 = default) used by the last batch        */
  int32_t tuned_vfuse;  /* V-cycle form of the last batch: 1 fused, 0 per step,
                           -1 the params.vfuse rule                              */
  double vcycle_ms;
  int64_t vcycle_count;
  int64_t vcycle_bytes;
} lcmg_stats;
int lcmg_get_stats(lcmg_ctx* ctx, lcmg_stats* out);

/* Apply K = A^T A + lambda^2 L^T D^2 L to n_cols device vectors
 * x_dev[n_cols][n] -> y_dev[n_cols][n] in FP64 (one lambda per column). */
int lcmg_apply_normal_dev(lcmg_ctx* ctx, int32_t n_cols, const double* lambda,
                          const double* x_dev, double* y_dev);

/* Apply one V-cycle z = B(lambda) r to n_cols device vectors (FP64 or the
 * context's precision), r_dev, z_dev laid out [n_cols][n]. */
int lcmg_apply_vcycle_dev(lcmg_ctx* ctx, int32_t n_cols, const double* lambda,
                          const double* r_dev, double* z_dev);

/* Copy the Galerkin coarse operators of level k >= 1 to the host: 25
 * coefficient arrays per part, gl[25][n_k] and ga[25][n_k], offset index
 * (di + 2) + 5 (dj + 2) for the neighbour (i + di, j + dj).  Level 0 is the
 * 5-point fine operator.  Returns the level's n_v, n_h. */
int lcmg_get_level(lcmg_ctx* ctx, int32_t k, int32_t* n_v, int32_t* n_h, double* gl,
                   double* ga);

/* Number of multigrid levels of the current hierarchy. */
int lcmg_num_levels(lcmg_ctx* ctx, int32_t* levels);

/* diag(A^T A) (n doubles, host). */
int lcmg_get_diag(lcmg_ctx* ctx, double* diag_out);

/* Measured arithmetic peak (TFLOP/s, multiply-add = 2 flops) of the FP64
 * (precision = LCMG_PREC_FP64) or FP32 (LCMG_PREC_MIXED) pipe of device
 * `device`: independent multiply-add chains on every SM, best of 5 timed
 * launches.  A measurement utility that bounds the FP64 kernels of this
 * library (the paper has no counterpart).  Errors: INVALID_ARG, CUDA. */
int lcmg_fma_peak(int device, int32_t precision, double* tflops);

/* Allocation-free application of q_j = (A^T A + lambda_j^2 L^T D^2 L) p_j.
 * The paper has no counterpart: this exists for callers that cannot
 * allocate device memory where they need the operator (code under an
 * external memory manager that owns every device byte, a real-time loop
 * that cannot pay an allocation's synchronisation, a thread that must not
 * enter the allocator).  Unlike lcmg_apply_normal_dev it needs no context
 * and calls no cudaMalloc/cudaFree: every input and output is a
 * caller-owned device pointer on `device`, and the intermediate A p lives
 * in a fixed array of 2^19 doubles (4 MiB) in the library's device image,
 * held by every GPU that loads the library until the process exits.
 *   device, stream   CUDA device of all pointers; stream (cudaStream_t) the
 *                    two kernels are launched on; the call does not
 *                    synchronise.  The caller's current device is restored.
 *   n_v, n_h, m      image grid and the number of rows of A
 *   row_ptr[m+1], col[nnz], val[nnz]          A as CSR (int64, int32, values)
 *   row_ptr_t[n+1], col_t[nnz], val_t[nnz]    A^T as CSR (n = n_v n_h)
 *   val_dtype        0 = FP32 values, 1 = FP64 values (both matrices)
 *   d[n_edges]       edge weights D, ordered as in lcmg_set_weights
 *   n_cols           columns, 1..64, with n_cols * m <= 2^19
 *   lambda[n_cols]   host array
 *   p, q             [n_cols][n] device arrays (each column contiguous)
 * Preconditions the library cannot check on the device: 0 <= col < n and
 * 0 <= col_t < m; (row_ptr_t, col_t, val_t) is the transpose of the m-row A
 * given by (row_ptr, col, val), with m its true row count; every pointer is
 * valid for the sizes above.  p and q must not overlap (q is written while
 * neighbouring entries of p are read; checked on the host).
 * Arithmetic is FP64.  Every call looks up the array's device address in
 * the current context (cudaGetSymbolAddress, with `device` current; no
 * allocation).  The first call on a device loads the library's device image
 * there if it is not loaded yet, which commits the 4 MiB array on that
 * device: make that first call before any stream capture.  Every call
 * shares the one array and overwrites what it reads, so calls whose kernels
 * overlap on the GPU (other streams, other threads) race: order them.
 * Errors: INVALID_ARG (sizes, null pointers, p and q overlapping, n_cols * m
 * above the limit), CUDA. */
int lcmg_apply_normal_noalloc(int device, void* stream, int32_t n_v, int32_t n_h, int64_t m,
                              const int64_t* row_ptr, const int32_t* col, const void* val,
                              const int64_t* row_ptr_t, const int32_t* col_t, const void* val_t,
                              int32_t val_dtype, const double* d, int32_t n_cols,
                              const double* lambda, const double* p, double* q);

/* ---- serving ----------------------------------------------------------
 * A server keeps forward operators ("problems") resident on one device and
 * runs the requests submitted against them, each a lambda sweep (the
 * systems of eq. (normal) for a list of lambda, Sec. 4) or a whole
 * Algorithm 2 run, on up to max_slots slots.  A slot is a host thread that
 * drives its own context (own CUDA stream, operator copy, hierarchy and
 * workspace), so requests running in different slots overlap on the
 * device.  Admission: in arrival order among the requests that fit, as soon
 * as a slot is free and the request's device bytes fit in hbm_budget_bytes
 * next to everything resident.  An idle context of the same problem is
 * reused (operator, hierarchy and its last solutions stay resident; a
 * request with warm = 1 and the same lambda list starts from them);
 * otherwise a context is created, evicting idle contexts least recently
 * used.  A request larger than the whole budget fails with NOMEM.  Each
 * request computes what lcmg_solve / lcmg_lcurve_run compute on a fresh
 * context with the server's params (same kernels, same reduction order),
 * whatever else runs.  The paper has no counterpart: this is the service
 * form of its lambda sweep.  All calls are thread-safe. */
typedef struct lcmg_server lcmg_server;

typedef struct {
  int32_t n_v, n_h;          /* image grid (defines L)                         */
  int32_t kind;              /* 0: CSR matrix A; 1: PSF stencil                 */
  int64_t m;                 /* CSR: rows of A                                 */
  const int64_t* row_ptr;    /* CSR, copied: m + 1                             */
  const int32_t* col;        /* CSR, copied: nnz                               */
  const void* val;           /* CSR, copied: nnz FP32 (val_dtype 0) or FP64 (1) */
  int32_t val_dtype;
  int32_t kh, kw;            /* PSF: odd sides                                  */
  const double* psf;         /* PSF, copied: kh x kw row-major                  */
} lcmg_problem;

typedef struct {
  int32_t problem;           /* id from lcmg_server_add_problem                 */
  int32_t n_lambda;
  const double* lambda;      /* increasing, > 0; copied at submit               */
  const double* b;           /* m values (n for a PSF problem); copied          */
  double tol;                /* relative residual; 0 = the server's params.tol   */
  int32_t max_outer;         /* 0: one sweep over lambda (D = I);
                                >= 1: Algorithm 2 with at most this many outer
                                iterations (needs n_lambda >= 3)                */
  int32_t warm;              /* sweep: 1 = start from the resident solutions of
                                the last sweep of the same problem and lambda
                                list on the reused context, if any             */
} lcmg_request;

typedef struct {
  int32_t state;             /* lcmg_status of the request (OK, NOMEM, CUDA, ...) */
  int32_t n_lambda;
  int32_t n_outer;           /* Algorithm 2: outer iterations run               */
  int64_t n_solves, n_converged;
  double t_submit, t_admit, t_done;  /* seconds, the server's monotonic clock  */
  /* caller-owned outputs (each may be NULL), written by poll / wait:
     sweep:        x[n_lambda][n], rho, eta[n_lambda], iters, status[n_lambda]
     Algorithm 2:  x[n] (the selected solution), history[max_outer]          */
  double* x;
  double* rho;
  double* eta;
  int32_t* iters;
  int32_t* status;
  int32_t* history;
} lcmg_result;

typedef struct {
  size_t resident_bytes;     /* device bytes counted against the budget         */
  int32_t contexts, pending, running, peak_running;
  int64_t admitted, completed, evictions, reuses;
} lcmg_server_stats;

/* Start a server on `device` with max_slots (1..64) slot threads; p = NULL
 * takes lcmg_default_params.  Errors: INVALID_ARG, CUDA (no such device). */
int lcmg_server_create(lcmg_server** out, int device, size_t hbm_budget_bytes, int32_t max_slots,
                       const lcmg_params* p);
/* Register a forward operator; *id identifies it in requests.  INVALID_ARG. */
int lcmg_server_add_problem(lcmg_server* s, const lcmg_problem* pr, int32_t* id);
/* Queue a request; returns at once with its ticket.  INVALID_ARG. */
int lcmg_server_submit(lcmg_server* s, const lcmg_request* rq, uint64_t* ticket);
/* NOT_READY while the request is queued or running; CANCELLED if it was
 * cancelled; otherwise OK with out filled (out->state is the request's own
 * outcome).  A ticket is released once OK or CANCELLED has been returned. */
int lcmg_server_poll(lcmg_server* s, uint64_t ticket, lcmg_result* out);
/* As poll but blocks until the request ends or timeout_s (<= 0: no limit)
 * passes (then NOT_READY). */
int lcmg_server_wait(lcmg_server* s, uint64_t ticket, double timeout_s, lcmg_result* out);
/* Cancel a queued request (STATE if it already started). */
int lcmg_server_cancel(lcmg_server* s, uint64_t ticket);
int lcmg_server_get_stats(lcmg_server* s, lcmg_server_stats* out);
/* Estimated device bytes of a context of `problem` solving n_cols columns
 * (what admission counts). */
int lcmg_server_footprint(lcmg_server* s, int32_t problem, int32_t n_cols, size_t* bytes);
/* Message of the calling thread's last server failure. */
const char* lcmg_server_last_error(void);
/* Cancel queued requests, let running ones finish, free everything. */
int lcmg_server_destroy(lcmg_server* s);

#ifdef __cplusplus
}
#endif
#endif /* LCMG_H */
