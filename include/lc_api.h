/*
 * lc_api.h -- C ABI of the GB300 (sm_103a) library for the local
 * character-based linear solve of Ye, An & Xu, "A local character based
 * method for solving linear systems of radiation diffusion problems"
 * (arXiv 2001.01158).
 *
 * The problem (Sec. 2.1): solve A x = b, A in R^{N x N} sparse, from an
 * initial iterate x0 (the previous time step or nonlinear iterate), by
 *   1. marking a local domain Omega_local of "bad points" (Alg 2 from the
 *      gradient of x0, or Alg 3 from the residual of x0),
 *   2. extracting and solving the local subsystem B x_B = b_B - E x_C^(0)
 *      (Eq. loc-equ), assembling x~ (Eq. sol-assemble),
 *   3. returning x~ if it meets ||b - A x~||_2 <= eps ||b||_2 (Eq.
 *      rel-res-conv-criteria), else solving the whole system from x~
 *      (Alg 1).  The Krylov solver is Jacobi-preconditioned CG.
 *
 * Conventions shared by every entry point:
 *   - Every pointer argument named as a vector or array is a DEVICE pointer
 *     on the context's device unless stated otherwise; the caller owns it
 *     and keeps it alive until the work enqueued on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work and return without waiting, except that
 *     a call given a non-NULL host `lc_stats*` waits for its stream before
 *     filling it.
 *   - Operators (lc_op) keep the caller's coefficient pointers (no copy) and
 *     own workspaces sized at creation for N and nnz(A); no entry point
 *     below allocates device memory.
 *   - Vectors are FP64, indices int32, masks uint8 (0 or 1); cell index of a
 *     structured grid i = x + nx*(y + ny*z).
 *   - Return value: LC_OK or an lc_status code; on error the outputs are
 *     unspecified except for LC_ERR_NOT_CONVERGED (x holds the last iterate
 *     and stats are filled).  lc_last_error() gives a message.
 *   - Calls on one context must not overlap in time from several host
 *     threads; work on one operator must be serialised on one stream (the
 *     operator's workspaces are shared by its calls).
 */
#ifndef LC_API_H
#define LC_API_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LC_API_VERSION 1

#if defined(__GNUC__)
#define LC_EXPORT __attribute__((visibility("default")))
#else
#define LC_EXPORT
#endif

typedef struct lc_ctx lc_ctx;
typedef struct lc_op lc_op;

typedef enum {
    LC_OK = 0,
    LC_ERR_INVALID_ARG = 1,    /* null pointer, bad size, unsorted CSR, non-positive diagonal, bad mode */
    LC_ERR_CUDA = 2,           /* a CUDA runtime call failed (message in lc_last_error) */
    LC_ERR_NO_MEMORY = 3,      /* workspace allocation at creation failed */
    LC_ERR_NOT_CONVERGED = 4,  /* max_iter reached; x = last iterate */
    LC_ERR_BREAKDOWN = 5,      /* p^T A p <= 0 or not finite (A not SPD, or NaN input) */
    LC_ERR_TIMEOUT = 6,        /* a bounded grid-wide wait inside a persistent kernel gave up */
    LC_ERR_TOO_LARGE = 7,      /* sizes beyond int32 indexing or the documented limits */
    LC_ERR_UNSUPPORTED = 8     /* valid request the library does not provide */
} lc_status;

/* Threshold of the residual marking. */
enum {
    LC_THR_EPS_NORMB = 0,  /* tau = eps ||b||_2 / sqrt(N)  (Sec. 2.3.1)  */
    LC_THR_REL_MAX = 1     /* tau = beta * max_i |r0_i|   (relative variant) */
};
/* Expansion of the residual-marked set. */
enum {
    LC_EXP_NONE = 0,
    LC_EXP_DILATE = 1,     /* add every neighbour, `rounds` times (graph layers) */
    LC_EXP_PAPER = 2       /* Alg 3: at most `rounds` = E_max conditional rounds */
};
enum { LC_MARK_RESIDUAL = 0, LC_MARK_GRADIENT = 1 };
enum { LC_PREC_FP64 = 0, LC_PREC_MIXED = 1 };

/* Residual-marking parameters (Alg 3 and its relative/dilation variant). */
typedef struct {
    int32_t thr_mode;    /* LC_THR_* */
    double  thr_param;   /* eps (LC_THR_EPS_NORMB) or beta (LC_THR_REL_MAX), >= 0 */
    int32_t exp_mode;    /* LC_EXP_* */
    int32_t exp_rounds;  /* layers (DILATE) or E_max (PAPER), 0..64 */
} lc_mark_params;

/* Krylov solve parameters. */
typedef struct {
    double  tol;         /* stop when ||b - A x||_2 <= tol ||b||_2 (Eq. rel-res-conv-criteria) */
    int32_t max_iter;    /* total CG iterations (all refinement sweeps together) */
    int32_t precision;   /* LC_PREC_FP64, or LC_PREC_MIXED: FP32 inner CG, FP64 refinement */
    double  inner_tol;   /* MIXED: relative reduction asked of each FP32 inner solve (e.g. 1e-5); a
                            sweep that needs less asks for half of what the outer test still misses */
    int32_t max_outer;   /* MIXED: refinement sweeps (e.g. 20) */
} lc_solve_params;

/* Alg 1 parameters. */
typedef struct {
    int32_t         mark_mode;    /* LC_MARK_RESIDUAL | LC_MARK_GRADIENT */
    lc_mark_params  mark;         /* residual marking */
    double          alpha;        /* gradient marking (Alg 2), in [0, 1] */
    int32_t         grad_layers;  /* dilation layers after Alg 2 (0 = as printed) */
    lc_solve_params global;       /* the whole-system solve (Alg 1 step 11) */
    lc_solve_params local;        /* the subsystem solve (Alg 1 step 5); tol relative to ||rhs_L||_2 */
    int32_t         gs_sweeps;    /* Gauss-Seidel sweeps of Alg 1 step 7 on x~, 0..64 (see lc_gs_smooth) */
} lc_params;

/* Per-call statistics in the paper's notation (Sec. 3: N, K, eta = K/N). */
typedef struct {
    int32_t status;         /* lc_status of the call */
    int32_t n;              /* N */
    int32_t K;              /* |Omega_local| */
    int32_t nnzB;           /* nnz of the local block B */
    int32_t it_local;       /* CG iterations of the subsystem solve */
    int32_t it_global;      /* CG iterations of the whole-system solve (0 if x~ was accepted) */
    int32_t early_exit;     /* 1 if x~ met the criterion (Alg 1 step 9) */
    int32_t restarts;       /* true-residual restarts / refinement sweeps of the global solve */
    double  tau;            /* marking threshold (or g_max for gradient marking) */
    double  eta;            /* K / N */
    double  relres_tilde;   /* ||b - A x~|| / ||b|| */
    double  relres_final;   /* ||b - A x|| / ||b|| on return */
    float   t_mark_ms, t_extract_ms, t_local_ms, t_global_ms, t_total_ms;  /* CUDA-event phase times */
} lc_stats;

/* Caller-allocated outputs of lc_extract (device pointers).  Capacities:
 * g2l[N], l2g[N], rowptr[N+1], col[nnz(A)], val[nnz(A)], rhs[N], xL0[N],
 * K[1], nnz[1].  Only the first K (resp. K+1, nnzB) entries are written. */
typedef struct {
    int32_t *g2l;     /* global -> local index, -1 outside Omega_local */
    int32_t *l2g;     /* local -> global, ascending global order */
    int32_t *rowptr;  /* CSR of B = A[Omega, Omega] in local indices */
    int32_t *col;
    double  *val;     /* copied bit for bit from A */
    double  *rhs;     /* b_B - E x_C^(0) (Eq. loc-equ), canonical order (below) */
    double  *xL0;     /* x0 restricted to Omega_local */
    int32_t *K;       /* device scalar: K */
    int32_t *nnz;     /* device scalar: nnz(B) */
} lc_subsys;

/* ---- context and operators ------------------------------------------- */

/* Create a context on CUDA device `device` (sets it current for the call).
 * lc_ctx_destroy releases the caller's handle; operators and batches created
 * on the context keep it alive until they are destroyed too, so the handles
 * may be destroyed in any order (the context's memory is freed with the last
 * of them).  Using a context handle after lc_ctx_destroy is an error. */
LC_EXPORT int lc_ctx_create(lc_ctx **ctx, int device);
LC_EXPORT int lc_ctx_destroy(lc_ctx *ctx);

/* General sparse A (CSR, device pointers): rowptr[n+1], col[nnz] ascending
 * and unique within each row, val[nnz]; every row must hold its diagonal
 * with a positive value (checked; LC_ERR_INVALID_ARG otherwise).
 * nnz < 2^31 (LC_ERR_TOO_LARGE).  The neighbours of i are the j != i with a
 * stored a_ij != 0. */
LC_EXPORT int lc_op_create_csr(lc_ctx *ctx, lc_op **op, int32_t n, int64_t nnz,
                     const int32_t *rowptr, const int32_t *col, const double *val);

/* Structured 5-point (dim 2) or 7-point (dim 3) operator, shape = {nx, ny,
 * nz} (nz = 1 for dim 2), device arrays of N = nx*ny*nz values:
 *   D  diagonal a_ii > 0
 *   Tx face conductance between i and i+1     : a_{i,i+1} = a_{i+1,i} = -Tx[i]
 *   Ty face conductance between i and i+nx    : a_{i,i+nx} = -Ty[i]
 *   Tz face conductance between i and i+nx*ny : (dim 3 only; NULL for dim 2)
 * Every interior face conductance must be > 0 (checked); entries on the last
 * column/row/plane are not read.  This is the same matrix, bit for bit, as
 * the CSR with those negated entries in ascending column order. */
LC_EXPORT int lc_op_create_stencil(lc_ctx *ctx, lc_op **op, int32_t dim, const int32_t shape[3],
                         const double *D, const double *Tx, const double *Ty, const double *Tz);
LC_EXPORT int lc_op_destroy(lc_op *op);

/* ---- the hot path ------------------------------------------------------- */

/* Residual-based local domain (Alg 3; Eq. resi-local-domain-0).
 *   r0 = b - A x0 with r_i = b_i; r_i = fma(-a_ij, x0_j, r_i) over j
 *   ascending (the canonical order; bit-identical for stencil and CSR).
 *   tau: EPS_NORMB: (eps*sqrt(S))/sqrt((double)N), S = sum b_i^2 by a
 *   stride-halving tree over zero-padded chunks of 1024, repeated on the
 *   chunk sums; REL_MAX: beta * max_i |r0_i| (NaN entries ignored).
 *   mask_i = |r0_i| > tau, then the expansion: DILATE adds all neighbours
 *   `rounds` times; PAPER runs Alg 3's synchronous rounds with
 *   c_j = |r0_j| + t, t = sum over domain neighbours i (ascending) of
 *   |a_ji * x0_i| (one rounded product, then a rounded sum), added if c_j > tau.
 * Outputs: mask[N]; r0_opt[N] (may be NULL); K_dev[1] = |Omega_local|;
 * tau_dev[1] (may be NULL).  The results are bit-identical to a serial FP64
 * evaluation of these definitions. */
LC_EXPORT int lc_mark_residual(lc_ctx *ctx, const lc_op *op, const double *b, const double *x0,
                     const lc_mark_params *p, uint8_t *mask, double *r0_opt,
                     int32_t *K_dev, double *tau_dev, void *stream);

/* Gradient-based local domain (Alg 2; Eq. grad): g_i = sum over neighbours
 * j (ascending) of |x0_i - x0_j| (plain additions from 0), g_max = max(0,
 * max g), mask_i = g_i > fl(alpha * g_max), then `layers` dilation rounds.
 * Outputs mask[N], K_dev[1], gmax_dev[1] (may be NULL). */
LC_EXPORT int lc_mark_gradient(lc_ctx *ctx, const lc_op *op, const double *x0, double alpha, int32_t layers,
                     uint8_t *mask, int32_t *K_dev, double *gmax_dev, void *stream);

/* Local subsystem (Sec. 2.1, Eq. loc-equ) from a mask: local indices in
 * ascending global order; B = A[Omega, Omega] with values copied; rhs_l =
 * b_i; rhs_l = fma(-a_ij, x0_j, rhs_l) over non-local j ascending; xL0 =
 * x0[Omega].  Bit-identical to the serial definition. */
LC_EXPORT int lc_extract(lc_ctx *ctx, const lc_op *op, const uint8_t *mask, const double *b,
               const double *x0, const lc_subsys *out, void *stream);

/* Jacobi-preconditioned CG on the whole system from the iterate in x (in:
 * x0, out: x).  Stops when ||r||^2 <= tol^2 ||b||^2 on the recurrence
 * residual, then confirms with the true residual and restarts from it if
 * needed (at most 3 restarts).  b = 0 gives x = 0.  One persistent
 * cooperative launch (FP64), or FP32 inner solves inside FP64 iterative
 * refinement (LC_PREC_MIXED).  stats (host, may be NULL) waits for the
 * stream. */
LC_EXPORT int lc_pcg_solve(lc_ctx *ctx, const lc_op *op, const double *b, double *x,
                 const lc_solve_params *p, lc_stats *stats, void *stream);

/* Gauss-Seidel smoothing (Alg 1 step 7): `sweeps` (0..64) multicolour
 * Gauss-Seidel sweeps over the whole system A x = b, in place in x (device,
 * N values).  Colour after colour, every point i of the colour is set to
 *     s = b_i; for j ascending, j != i: s = fma(-a_ij, x_j, s); x_i = s / a_ii
 * from the newest neighbour values.  Stencil operators use the red-black
 * colouring (x + y + z) mod 2; CSR operators need lc_op_set_colouring first
 * (else LC_ERR_UNSUPPORTED).  Since no two neighbours share a colour, the
 * result equals the serial sweep bit for bit. */
LC_EXPORT int lc_gs_smooth(lc_ctx *ctx, const lc_op *op, const double *b, double *x, int32_t sweeps,
                           void *stream);

/* Colouring of a CSR operator's rows for lc_gs_smooth: colour[n] (device,
 * uint8, values < ncolours, kept by reference like the operator's arrays),
 * checked on the device to give no two neighbours (stored a_ij != 0, j != i)
 * the same colour (LC_ERR_INVALID_ARG otherwise; waits for the check).
 * colour = NULL removes it.  Stencil operators: LC_ERR_INVALID_ARG. */
LC_EXPORT int lc_op_set_colouring(lc_op *op, const uint8_t *colour, int32_t ncolours);

/* Alg 1 without host synchronisation: mark (residual or gradient), extract,
 * local Jacobi-PCG from xL0 (tolerance relative to ||rhs||), assemble x~ in
 * place in x, smooth it by p->gs_sweeps Gauss-Seidel sweeps (lc_gs_smooth),
 * check ||b - A x~|| <= tol ||b||, and only if that fails run the global PCG
 * from x~.  x: in x0, out x.  stats (host, may be NULL) waits for the stream
 * and fills phase times (t_local_ms includes assembly and smoothing). */
LC_EXPORT int lc_solve_local_then_global(lc_ctx *ctx, const lc_op *op, const double *b, double *x,
                               const lc_params *p, lc_stats *stats, void *stream);

/* ---- many independent systems in one launch -----------------------------------
 *
 * Alg 1 on a batch of independent 2D 5-point systems of uneven sizes (each
 * system its own nx x ny grid), all solved by ONE persistent kernel launch in
 * which each CTA takes systems from a device work queue (largest first) and
 * runs the whole method on one system with block-level synchronisation:
 * residual marking (relative threshold, layer dilation), extraction,
 * local solve and the check/global solve, both as FP32 Jacobi-CG inside
 * FP64 iterative refinement.  The launch can be captured once into a CUDA
 * graph and replayed.  Masks and subsystems are bit-identical to
 * lc_mark_residual / lc_extract on each system; the solves reach the FP64
 * relative residual `global.tol`. */
typedef struct lc_batch lc_batch;

/* nx[nsys], ny[nsys] are HOST arrays; D, Tx, Ty are DEVICE arrays holding
 * the systems' stencil coefficients concatenated in system order (system s
 * occupies cells [sum_{t<s} nx_t ny_t, ...) in the layout of
 * lc_op_create_stencil).  Allocates the batch's workspace (about 160 bytes
 * per cell) and FP32 copies of the coefficients; synchronises the device.
 * The caller keeps D, Tx, Ty alive and unchanged while the batch is used. */
LC_EXPORT int lc_batch_create(lc_ctx *ctx, lc_batch **batch, int32_t nsys, const int32_t *nx, const int32_t *ny,
                              const double *D, const double *Tx, const double *Ty);
LC_EXPORT int lc_batch_destroy(lc_batch *batch);

/* Enqueue one batched solve: b (device, concatenated) and x (device; in x0,
 * out x).  p must ask for residual marking with LC_THR_REL_MAX, LC_EXP_NONE
 * or LC_EXP_DILATE, and LC_PREC_MIXED for both solves (otherwise
 * LC_ERR_UNSUPPORTED); global.max_iter caps each inner FP32 solve,
 * global.max_outer the refinement sweeps, local.tol is relative to the
 * subsystem's right-hand side. */
LC_EXPORT int lc_batch_solve(lc_ctx *ctx, lc_batch *batch, const double *b, double *x, const lc_params *p,
                             void *stream);

/* Capture the same work (for these b, x and p) into a CUDA graph held by the
 * batch, on a stream of the library's own; lc_batch_replay launches it on
 * `stream`.  A new capture replaces the previous graph. */
LC_EXPORT int lc_batch_capture(lc_ctx *ctx, lc_batch *batch, const double *b, double *x, const lc_params *p);
LC_EXPORT int lc_batch_replay(lc_batch *batch, void *stream);

/* Waits for `stream`, then fills per_system[nsys] (host): status, n, K, nnzB,
 * it_local, it_global (FP32 inner iterations), restarts (= refinement sweeps
 * of the global solve), early_exit, tau, eta, relres_tilde, relres_final.
 * Returns the first non-OK system status, else LC_OK. */
LC_EXPORT int lc_batch_stats(lc_batch *batch, lc_stats *per_system, void *stream);

/* The local domain and subsystem of system `sys` (0 .. nsys-1) from the
 * last lc_batch_solve / lc_batch_replay, for inspection: waits for `stream`,
 * then copies into caller DEVICE buffers (each may be NULL to skip it)
 *   mask[n]        the final mask (0/1) after thresholding and dilation
 *   g2l[n]         local index of each cell, -1 outside the domain
 *   l2g[K]         cell of each local index (ascending)
 *   rowptr[K+1], col[nnzB], val[nnzB]   B = A[Omega, Omega] in local indices
 *   rhs[K]         b_B - E x_C^(0) in the canonical order (Eq. loc-equ)
 * with n = nx[sys] ny[sys] and K, nnzB as lc_batch_stats reports them.
 * These are the same bits lc_mark_residual and lc_extract produce for the
 * system (Sec. 2.3, Eq. loc-equ).  The subsystem's starting values x0[Omega]
 * are not kept (the local solve overwrites them).  Synchronous; invalid
 * `sys` returns LC_ERR_INVALID_ARG. */
LC_EXPORT int lc_batch_domain(lc_batch *batch, int32_t sys, uint8_t *mask, int32_t *g2l, int32_t *l2g,
                              int32_t *rowptr, int32_t *col, double *val, double *rhs, void *stream);

/* Launch-shape knobs (for the autotuner): "block" = 256 | 512 | 1024 threads
 * per CTA (default 512); "ctas_per_sm" = 0 (as many as fit) .. 32;
 * "cluster" = 1 | 2 | 4 | 8 | 16 CTAs per thread-block cluster (default 1: every
 * system on one CTA); "big_cells" (default 65536): with clusters, every
 * system of at least this many cells is solved by a whole cluster (its rows
 * split among the cluster's CTAs), the others by one CTA each.  Results do
 * not depend on the knobs beyond the rounding order of the solves' sums. */
LC_EXPORT int lc_batch_set_tuning(lc_batch *batch, const char *key, int32_t value);

/* ---- operators from conductivity, and the adjoint -----------------------------
 *
 * 2D backward-Euler diffusion on an nx x ny grid (grid units):
 *   A(k) = I/dt + sum_faces T_f (e_P - e_N)(e_P - e_N)^T + sum_{boundary faces} 2 k_P e_P e_P^T,
 *   T_f = 2 k_P k_N / (k_P + k_N)  (harmonic face conductance; homogeneous
 *   Dirichlet ghost half a cell outside each boundary face),
 * the operator family of the paper's time-stepped diffusion systems (Sec. 3).
 * These calls make the solve differentiable: for a loss L(x), x = A(k)^-1 b,
 * the adjoint lambda = A^-T dL/dx (A is symmetric, so any solve of this
 * library computes it) gives dL/db = lambda and dL/dk per cell (below). */

/* D, Tx, Ty (device, N = nx*ny each, stencil layout of lc_op_create_stencil)
 * from per-cell conductivities k[N] > 0 and dt > 0.  Per cell, in this
 * order: T = ((2 kP) kE) / (kP + kE) for each interior face; D = 1/dt + east
 * + west + north + south face conductances + 2 kP for each boundary face
 * (west, east, south, north).  Tx/Ty on the last column/row are set to 0. */
LC_EXPORT int lc_assemble_diffusion_2d(lc_ctx *ctx, const int32_t shape[2], const double *k, double dt, double *D,
                                       double *Tx, double *Ty, void *stream);

/* Recompute an operator's derived data (1/D and the FP32 copies used by
 * LC_PREC_MIXED) after its coefficient arrays were changed in place, e.g.
 * by lc_assemble_diffusion_2d.  Stream-ordered; the new coefficients are not
 * re-validated (they must keep D > 0 and interior faces > 0).  No-op for CSR
 * operators (their derived data is formed per solve). */
LC_EXPORT int lc_op_refresh(lc_op *op, void *stream);

/* dk[c] = dL/dk_c = - sum_{interior faces (c,N)} 2 k_N^2/(k_c+k_N)^2 (lam_c - lam_N)(x_c - x_N)
 *                   - sum_{boundary faces of c} 2 lam_c x_c
 * for the operator of lc_assemble_diffusion_2d, given the state x and the
 * adjoint lam (A lam = dL/dx).  Derived from dL/dk = -lam^T (dA/dk) x.  All
 * arrays device, N values. */
LC_EXPORT int lc_adjoint_grad_k_2d(lc_ctx *ctx, const int32_t shape[2], const double *k, const double *x,
                                   const double *lam, double *dk, void *stream);

/* The whole backward step of x = A(k)^-1 b in one call, for a loss L(x)
 * with gradient gx = dL/dx at the forward solution x:
 *   1. A(k) is assembled again from k and dt into the operator's own
 *      coefficient arrays (lc_assemble_diffusion_2d + lc_op_refresh): no
 *      state of the forward solve is kept;
 *   2. lambda solves A lambda = gx by Alg 1 with parameters p (A is
 *      symmetric, so this is the adjoint A^T lambda = dL/dx); lambda holds
 *      the starting iterate on entry (e.g. zeros) and dL/db on return;
 *   3. dk = dL/dk per cell by lc_adjoint_grad_k_2d.
 * op must be a 2D stencil operator created on the D, Tx, Ty arrays that
 * lc_assemble_diffusion_2d fills for this grid (the call rewrites them with
 * the same values for the same k and dt); k, x, gx, lambda, dk are device
 * arrays of N values.  stats (host, may be NULL) are the adjoint solve's and
 * wait for the stream; errors as lc_solve_local_then_global.  The paper has
 * no adjoint: this is the training form of the method's solve. */
LC_EXPORT int lc_adjoint_grad(lc_ctx *ctx, lc_op *op, const double *k, double dt, const double *x, const double *gx,
                              double *lambda, double *dk, const lc_params *p, lc_stats *stats, void *stream);

/* Self-test of the failure path of the grid-wide waits: a cooperative launch
 * of `blocks` blocks on the operator's control block whose barrier waits for
 * one arrival more than there are blocks, so it can only end by its limit
 * (limit_ms in (0, 2000]; the solvers' own limit is ~2 s).  Every block gives
 * up, records LC_ERR_TIMEOUT and returns: *status_out (host) receives the
 * recorded status (LC_ERR_TIMEOUT when the path works).  Nothing faults or
 * hangs, the context stays usable, and the control block is cleared
 * afterwards.  Waits for the device. */
LC_EXPORT int lc_selftest_barrier_timeout(lc_ctx *ctx, lc_op *op, int32_t blocks, double limit_ms,
                                          int32_t *status_out);

/* Reproducible dot product of two device vectors of the operator's size N:
 * *out (device) = sum_i x_i y_i, where every product x_i y_i is rounded once
 * to FP64, the products are added exactly as 128-bit integers relative to
 * the largest product's exponent (products more than 2^40 below it are
 * rounded at that resolution), and the total is rounded once (to nearest).
 * The result does not depend on the order of the additions or on the launch
 * configuration.  NaN if a product is not finite.  Uses the operator's
 * workspace: work on one operator stays serialised on one stream. */
LC_EXPORT int lc_op_dot(lc_ctx *ctx, const lc_op *op, const double *x, const double *y, double *out, void *stream);

/* ---- nonlinear 2D heat conduction (Sec. 3.2) --------------------------------
 *
 * dT/dt = div(kappa(T) grad T), kappa = T^p, on an nx x ny grid of square
 * cells of width h; backward Euler in time and Picard iteration (Eq.
 * picard-equs): T^{n+1,s+1} solves the linear system with kappa evaluated at
 * T^{n+1,s}.  The paper's test: 99 x 99 cells on the unit square, p = 3.5,
 * T = 1 at x = 0 and 1e-4 at x = 1, no flux at y = 0, 1, dt = 1e-2, linear
 * tolerance 1e-10, Picard until ||T^{s+1} - T^s||_2 < 1e-8. */
enum { LC_BC_DIRICHLET = 0, LC_BC_NEUMANN = 1 };

/* Picard-linearised system from cell conductivities kappa (device, N) and
 * the previous time level Tn (device, N), as the 5-point stencil arrays of
 * lc_op_create_stencil (D, Tx, Ty, device, N each) and the right-hand side b
 * (device, N).  With c = 1/(h h), faces visited W, E, S, N:
 *   interior face T_f = ((2 kappa_P) kappa_N / (kappa_P + kappa_N)) c,
 *   Dirichlet side g = (2 kappa_P) c (ghost at half a cell), Neumann: none,
 *   D_P = 1/dt + each T_f or g in that order, Tx/Ty = T_f of the east/north
 *   face (0 on the last column/row), b_P = Tn_P (1/dt) + g T_side per
 *   Dirichlet side in that order.
 * bc_type[4] and bc_val[4] list the sides x-, x+, y-, y+. */
LC_EXPORT int lc_heat2d_assemble(lc_ctx *ctx, const int32_t shape[2], double h, double dt,
                                 const int32_t bc_type[4], const double bc_val[4], const double *kappa,
                                 const double *Tn, double *D, double *Tx, double *Ty, double *b, void *stream);

typedef struct {
    double    h;            /* cell width (> 0) */
    double    dt;           /* time step (> 0) */
    double    p;            /* kappa(T) = T^p */
    int32_t   bc_type[4];   /* sides x-, x+, y-, y+: LC_BC_* */
    double    bc_val[4];    /* Dirichlet values */
    int32_t   method;       /* 0: global Jacobi-PCG with params.global; 1: Alg 1 with params */
    lc_params params;
    double    picard_tol;   /* stop when ||T^{s+1} - T^s||_2 < picard_tol */
    int32_t   max_picard;   /* >= 1 */
} lc_heat2d_params;

typedef struct {
    int32_t picard_its;     /* Picard iterations of the step */
    int32_t it_local;       /* CG iterations of all local solves */
    int32_t it_global;      /* CG iterations of all global solves */
    int32_t K_sum;          /* sum of |Omega_local| over the step's solves */
    int32_t early_exits;    /* solves whose x~ met the criterion */
    int32_t status;         /* lc_status of the last solve */
    double  last_update;    /* ||T^{s+1} - T^s||_2 of the last iteration */
    float   t_solve_ms;     /* CUDA-event time of the linear solves */
    float   t_total_ms;     /* the whole step */
} lc_heat2d_stats;

/* One time step by Picard iteration: T (device, N) holds T^{n+1,0} on entry
 * (normally T^n) and T^{n+1} on exit; Tn (device, N) is T^n.  op must be the
 * 2D stencil operator created on D, Tx, Ty (device, N each), which this call
 * overwrites with each iteration's system (and refreshes the operator); b
 * (device, N) receives each right-hand side; work (device, 2N) is scratch.
 * Each iteration: kappa = T^p, assemble, solve from the previous iterate,
 * ||T^{s+1} - T^s||_2 (read on the host: the call waits for the stream).
 * stats (host) is filled. */
LC_EXPORT int lc_heat2d_step(lc_ctx *ctx, lc_op *op, const lc_heat2d_params *hp, const double *Tn, double *T,
                             double *D, double *Tx, double *Ty, double *b, double *work, lc_heat2d_stats *stats,
                             void *stream);

/* ---- kernel tuning ----------------------------------------------------------
 *
 * Launch-shape knobs of an operator's kernels, for the autotuner; not part
 * of the method (the paper has no counterpart).  Results do not depend on
 * them beyond the rounding order of the Krylov solve's reductions.
 *   "pcg_minblocks" 1..4 (default 3 for stencil operators, 4 for CSR):
 *       register budget of the persistent PCG kernels, as the number of
 *       256-thread blocks that must fit on an SM (2-D solves and local
 *       subsystem solves with pcg_big take one 768-thread block instead).
 *   "pcg_grid_cap"  0..4096 (default 0 = all that fit): blocks of the global
 *       PCG launch.
 *   "pcg_scaled"    0 or 1 (default 1): 2-D FP64 solves iterate on the
 *       symmetrically scaled system D^-1/2 A D^-1/2 (unit diagonal, so the
 *       Jacobi preconditioner becomes the identity) and map back, which is
 *       the same preconditioned iteration in exact arithmetic with fewer
 *       FP64 instructions and bytes per iteration.  0 iterates on A with the
 *       explicit Jacobi preconditioner.  The stopping test is the same in
 *       both: ||b - A x||_2 / ||b||_2 <= tol on the unscaled system.
 *   "pcg_wide"      0 or 1 (default 1): the scaled 2-D FP64 solve gives each
 *       lane four adjacent cells (else two) when nx is a multiple of 4.
 *   "pcg_big"       0 or 1 (default 1): 2-D solves (FP64 and mixed) and the
 *       local subsystem solves of lc_solve_local_then_global launch one block
 *       of 768 threads per SM instead of blocks of 256 (the same warps and
 *       register budget as pcg_minblocks 3, a third of the block partials
 *       and barrier arrivals per grid-wide reduction); pcg_minblocks then has
 *       no effect on them.  3-D solves and solves with a CSR operator's own
 *       matrix ignore it.
 *   "pcg_pairdot"   0 or 1 (default 1): the scaled 2-D (four cells per lane)
 *       and 3-D FP64 solves take their dot product p.q and the block sums
 *       of their grid reductions on pairs of FP32 numbers (hi + lo, 47
 *       significand bits, built from the FP64 bits with integer
 *       instructions; error-free FP32 products and two-sums) instead of on
 *       the FP64 pipe, which is the scarcer one on this GPU.  The vectors
 *       (x, r, p, q) stay FP64; alpha and beta differ from all-FP64 sums in
 *       rounding only.
 *   "pcg_lazy_x"    0 or 1 (default 1): with pcg_pairdot (2-D and 3-D), the update
 *       x += alpha_k p_k of iteration k is applied in iteration k+1's first
 *       phase, which loads p_k anyway (for p_k+1 = r + beta p_k), and after
 *       the last iteration by one extra pass: 8 fewer bytes per cell and
 *       iteration, the same operations in the same order (bit-identical x).
 *   "graph_max_cells" >= 0 (default 65536): for operators of at most this
 *       many unknowns, each lc_pcg_solve and lc_solve_local_then_global call
 *       runs as one CUDA graph, captured the first time a call signature is
 *       seen (the same b and x pointers, parameters, stats requested or not,
 *       and tuning) and replayed afterwards; its launches then reach the GPU
 *       together instead of one host call at a time (small systems are
 *       bound by that).  Every data-dependent decision of a solve is taken on
 *       the device, so a replay computes exactly what direct launches do.  If
 *       a capture fails, the operator launches directly from then on.  0
 *       disables it.
 *   "csr_store_p"   0 or 1 (default 1): the global solve of a CSR operator
 *       forms p = z + beta p_old once per row, stores it and, after one more
 *       grid barrier, reads it at the columns of the product; with 0 every
 *       entry recomputes p at its column (two loads and two FP64 FMAs per
 *       entry, no extra barrier).  The same arithmetic per value of p: the
 *       iterates are bit-identical.  Extracted subsystems always recompute. 
 *   "local_pipelined" 0 or 1 (default 1): the FP64 local solve of
 *       lc_solve_local_then_global on the whole grid runs pipelined CG (the
 *       Ghysels-Vanroose arrangement) on the symmetrically scaled subsystem
 *       diag(B)^-1/2 B diag(B)^-1/2 (Jacobi-PCG on B in exact arithmetic):
 *       one grid barrier per iteration, the iteration's sums read while the
 *       next product runs, and about 11 FP64 instructions per row and
 *       iteration instead of about 21.  In mixed precision the same
 *       arrangement, in FP32, is the inner solve of the FP64 iterative
 *       refinement.  Takes precedence over local_single.
 *   "local_single"  0 or 1 (default 0): the FP64 local solve of
 *       lc_solve_local_then_global takes one grid-wide reduction per CG
 *       iteration (Chronopoulos-Gear arrangement: same iterates in exact
 *       arithmetic) instead of two.
 *   "local_cluster_rows" >= 0 (default 2048): the FP64 local solve of
 *       lc_solve_local_then_global runs on one thread-block cluster, its
 *       vectors in distributed shared memory, when the subsystem has at most
 *       this many rows and they fit the cluster (about 76,000 rows on a
 *       GB300); larger subsystems, mixed precision, or 0 use the grid-wide
 *       kernel.  Same iteration, different rounding order of the dot
 *       products.  (Against the pipelined grid kernel the cluster is faster
 *       below about 1,000 rows and slower above about 3,000.)
 *   "local_cluster_threads" 256, 512 or 1024 (default 256): threads per CTA
 *       of that cluster.
 *   "local_cluster_ctas" 0, 2, 4, 8 or 16 (default 0 = the largest cluster the
 *       GPU schedules, 16 on a GB300): CTAs of that cluster.  Fewer CTAs give
 *       cheaper barriers and less FP64 throughput; a subsystem whose rows do
 *       not fit goes to the grid-wide kernel as before.
 *   "local_grid_cap" 0..4096 (default 0 = one block per SM): blocks of the
 *       grid-wide local solve kernel.
 * Unknown keys or out-of-range values return LC_ERR_INVALID_ARG. */
LC_EXPORT int lc_op_set_tuning(lc_op *op, const char *key, int32_t value);
LC_EXPORT int lc_op_get_tuning(const lc_op *op, const char *key, int32_t *value);

/* ---- marking without device allocation ------------------------------------
 *
 * For callers that cannot call cudaMalloc -- code that runs inside another
 * framework's memory pool or under a fixed memory budget, or a service that
 * must not allocate after start-up, and so cannot create an lc_op (whose
 * workspaces are allocated at creation).  The paper has no counterpart: this
 * is a deployment variant of lc_mark_residual.
 *
 * Same results, bit for bit, as lc_mark_residual on the stencil operator
 * (D, Tx, Ty, Tz, shape as in lc_op_create_stencil), but it allocates no
 * device memory: its scratch (control block, sum-of-squares tree partials,
 * second mask buffer of multi-pass expansion) is one fixed array of about
 * 4.3 MB compiled into the library, held by every device that loads the
 * library until the process exits.  The caller passes every input and
 * output: r0[N] is required (the residual is written there).
 *   - N = nx*ny*nz must not exceed LC_NOALLOC_MAX_CELLS: larger grids return
 *     LC_ERR_TOO_LARGE before any GPU work.
 *   - Null pointers, bad shapes or parameters return LC_ERR_INVALID_ARG; a
 *     failing CUDA call returns LC_ERR_CUDA.  There is no context, so no
 *     message is recorded.
 *   - The operator is not validated: interior face conductances must be > 0
 *     (the dilation uses the grid adjacency).
 *   - Every call looks up the scratch array's device address on the current
 *     device (host-side, no GPU work), so the address stays right after the
 *     device's context is reset.  The first call on a device also loads the
 *     library's device code there if nothing has loaded it yet; make that
 *     first call before any stream capture.
 *   - All calls share the one array, which keeps the previous call's
 *     contents; each call clears what must start at zero.  Calls that
 *     overlap on the GPU (other streams, other host threads) race on it and
 *     must be serialised by the caller. */
#define LC_NOALLOC_MAX_CELLS 4194304
LC_EXPORT int lc_mark_residual_stencil_noalloc(int32_t dim, const int32_t shape[3], const double *D,
                                               const double *Tx, const double *Ty, const double *Tz,
                                               const double *b, const double *x0, const lc_mark_params *p,
                                               uint8_t *mask, double *r0, int32_t *K_dev, double *tau_dev,
                                               void *stream);

/* ---- diagnostics ---------------------------------------------------------- */

LC_EXPORT const char *lc_error_string(int code);
LC_EXPORT const char *lc_last_error(const lc_ctx *ctx);

/* Number of CUDA kernels this library has launched in this process since it
 * was loaded (all contexts and devices; memsets and copies not counted).
 * For accounting only: a benchmark reads it before and after a timed region. */
LC_EXPORT int64_t lc_kernel_launch_count(void);

/* Bounds-checked builds only (the library compiled with -DLC_CHECKED, a
 * development build): every index the kernels take from data (CSR column
 * indices, the local domain's index maps) is tested against its range; a
 * failing index is replaced by a valid one and recorded.  This call waits
 * for nothing (synchronise first), collects and clears the records:
 * *failures (may be NULL) = the number of kernel files with a recorded
 * failure, `where` (len bytes, may be NULL) = "file:line" of the first.
 * Returns LC_OK, or LC_ERR_UNSUPPORTED in an ordinary build. */
LC_EXPORT int lc_checked_status(int32_t *failures, char *where, int32_t len);

/* Bounds-checked builds only: positive control of the checks.  Launches on
 * `stream` one thread that asks for element 4 of a 4-element device array
 * through the check; the check records the failure and substitutes element 0,
 * so nothing is accessed out of range.  After a synchronise,
 * lc_checked_status reports one failure in lc_api.cu.  Returns LC_OK,
 * LC_ERR_CUDA if the launch failed, or LC_ERR_UNSUPPORTED (launching
 * nothing) in an ordinary build. */
LC_EXPORT int lc_checked_selftest(void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LC_API_H */
