/*
 * lc_oracle.c -- plain, serial FP64 reference ("oracle") of the local
 * character-based linear solve of Ye, An & Xu, "A local character based
 * method for solving linear systems of radiation diffusion problems"
 * (arXiv 2001.01158).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or
 * call this file: it exists so that the tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA library with an obviously
 * correct, independent computation.  It shares no code with the CUDA path.
 *
 * Matrices are CSR with int32 row pointers and column indices sorted
 * ascending within each row, FP64 values.  Everything is a plain loop in
 * the paper's order; compiled with -ffp-contract=off so that the only fused
 * multiply-adds are the explicit fma() calls of the canonical orders below.
 *
 * Readings of points the paper leaves open (each is a fixed, documented
 * choice that the CUDA path must reproduce bit for bit where it decides a
 * set or a copied value):
 *   R1 residual (Alg 3 step 4, Eq. resi-local-domain-0):
 *        r_i = b_i; for j ascending: r_i = fma(-a_ij, x_j, r_i).
 *   R2 right-hand side of the local subsystem (Eq. loc-equ, b_B - E x_C):
 *        rhs = b_i; for j ascending with j outside the local domain:
 *        rhs = fma(-a_ij, x0_j, rhs).
 *   R3 ||b||_2^2 in the threshold eps*||b||_2/sqrt(N) (Sec. 2.3.1):
 *        squares b_i*b_i, summed by a stride-halving tree over zero-padded
 *        chunks of 1024, the chunk sums reduced again the same way until one
 *        value is left; tau = (eps*sqrt(S))/sqrt((double)N).
 *   R4 gradient mimic g_i (Eq. grad): terms |x_i - x_j| over stored entries
 *        with a_ij != 0 and j != i, ascending j, plain additions from 0.
 *   R5 neighbours of i: j != i with a stored a_ij != 0.
 *   R6 Alg 3 expansion quantity: t = 0; for i ascending in row j with i in
 *        the current local domain: t = t + |a_ji * x0_i|; c_j = |r_j| + t;
 *        all candidates of a round are tested against the domain as it was
 *        at the start of the round (synchronous update).
 *   R7 all thresholds are strict '>' (Alg 2, Alg 3).
 *   R8 local indices follow ascending global index (a symmetric
 *        permutation of the paper's Q; it leaves the subsystem's solution
 *        unchanged).
 *   R9 Gauss-Seidel smoothing (Alg 1 step 7): multicolour sweeps with a
 *        caller-given colouring in which no two neighbours share a colour;
 *        per point s = b_i; for j ascending, j != i: s = fma(-a_ij, x_j, s);
 *        x_i = s / a_ii.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Timing-only variant.  Built with -fopenmp (a separate library), the
 * row loops of the Krylov solve, the residual and the marking passes run in
 * parallel over rows and the dot products become OpenMP sum reductions
 * (another rounding order).  That build only times the method on all host
 * cores; the serial build below, without -fopenmp, is the parity oracle and
 * these macros expand to nothing there. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_ROWS _Pragma("omp parallel for schedule(static)")
#define ORC_ROWS_SUM _Pragma("omp parallel for schedule(static) reduction(+:s)")
#define ORC_ROWS_MAX _Pragma("omp parallel for schedule(static) reduction(max:mx)")
#else
#define ORC_ROWS
#define ORC_ROWS_SUM
#define ORC_ROWS_MAX
#endif

#define ORC_OK 0
#define ORC_NOT_CONVERGED 4
#define ORC_BREAKDOWN 5

/* ---------------------------------------------------------------- basics */

/* R1: r = b - A x  (Alg 3 step 4; Eq. resi-local-domain-0). */
void orc_residual(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                  const double *b, const double *x, double *r)
{
    ORC_ROWS
    for (int32_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
            s = fma(-av[e], x[ci[e]], s);
        r[i] = s;
    }
}

/* y = A x, plain sequential dot per row (used only inside the Krylov solve). */
static void spmv(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                 const double *x, double *y)
{
    ORC_ROWS
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
            s += av[e] * x[ci[e]];
        y[i] = s;
    }
}

static double dot(int32_t n, const double *a, const double *b)
{
    double s = 0.0;
    ORC_ROWS_SUM
    for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* R3: one level of the canonical tree -- sums of zero-padded chunks of 1024
 * values, each by stride halving (v[i] += v[i+s], s = 512, ..., 1). */
static int64_t tree_level(const double *in, int64_t n, double *out)
{
    double v[1024];
    int64_t nchunks = (n + 1023) / 1024;
    for (int64_t c = 0; c < nchunks; ++c) {
        for (int i = 0; i < 1024; ++i) {
            int64_t k = c * 1024 + i;
            v[i] = (k < n) ? in[k] : 0.0;
        }
        for (int s = 512; s >= 1; s >>= 1)
            for (int i = 0; i < s; ++i) v[i] = v[i] + v[i + s];
        out[c] = v[0];
    }
    return nchunks;
}

/* R3: S = sum_i b_i^2 in the canonical tree order. */
double orc_sumsq(int32_t n, const double *b)
{
    if (n <= 0) return 0.0;
    double *sq = (double *)malloc(sizeof(double) * (size_t)n);
    double *lv = (double *)malloc(sizeof(double) * (size_t)((n + 1023) / 1024 + 1));
    for (int32_t i = 0; i < n; ++i) sq[i] = b[i] * b[i];
    int64_t m = tree_level(sq, n, lv);
    while (m > 1) {
        int64_t m2 = tree_level(lv, m, sq);
        memcpy(lv, sq, sizeof(double) * (size_t)m2);
        m = m2;
    }
    double s = lv[0];
    free(sq);
    free(lv);
    return s;
}

/* Sec. 2.3.1: tau = eps * ||b||_2 / sqrt(N). */
double orc_tau_eps_normb(int32_t n, const double *b, double eps)
{
    double S = orc_sumsq(n, b);
    return (eps * sqrt(S)) / sqrt((double)n);
}

/* ------------------------------------------------------- marking (Sec. 2.3) */

/* R5 dilation: one round of mask_out = mask_in  U  neighbours(mask_in). */
static void dilate_once(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                        const uint8_t *in, uint8_t *out)
{
    ORC_ROWS
    for (int32_t i = 0; i < n; ++i) {
        uint8_t m = in[i];
        for (int32_t e = rp[i]; e < rp[i + 1] && !m; ++e)
            if (ci[e] != i && av[e] != 0.0 && in[ci[e]]) m = 1;
        out[i] = m;
    }
}

/* Unconditional expansion by `layers` graph layers. */
void orc_dilate(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                uint8_t *mask, int32_t layers)
{
    uint8_t *tmp = (uint8_t *)malloc((size_t)n + 1);
    for (int32_t l = 0; l < layers; ++l) {
        dilate_once(n, rp, ci, av, mask, tmp);
        memcpy(mask, tmp, (size_t)n);
    }
    free(tmp);
}

/* Alg 3 steps 10-23: at most emax expansion rounds.  Returns the number of
 * rounds that added points.  r0 holds the initial residual, x0 the initial
 * iterate, tau the threshold.  If c_trace is not NULL it receives, for round
 * m and point j, the tested quantity c_j (NaN where j was not a candidate);
 * it must hold emax*n values. */
int32_t orc_expand_paper(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                         const double *r0, const double *x0, double tau,
                         uint8_t *mask, int32_t emax, double *c_trace)
{
    if (c_trace)
        for (int64_t k = 0; k < (int64_t)emax * n; ++k) c_trace[k] = NAN;
    uint8_t *add = (uint8_t *)malloc((size_t)n + 1);
    int32_t rounds = 0;
    for (int32_t m = 0; m < emax; ++m) {
        int32_t k0 = 0;
        for (int32_t j = 0; j < n; ++j) {
            add[j] = 0;
            if (mask[j]) continue;
            int is_nbr = 0;
            double t = 0.0;
            for (int32_t e = rp[j]; e < rp[j + 1]; ++e) {
                int32_t i = ci[e];
                if (i == j || !mask[i]) continue;
                if (av[e] != 0.0) is_nbr = 1;
                t = t + fabs(av[e] * x0[i]);
            }
            if (!is_nbr) continue;          /* j is not a neighbour of the domain */
            double c = fabs(r0[j]) + t;
            if (c_trace) c_trace[(int64_t)m * n + j] = c;
            if (c > tau) { add[j] = 1; ++k0; }
        }
        if (k0 == 0) break;                 /* K0 = 0: nothing incorporated */
        for (int32_t j = 0; j < n; ++j) if (add[j]) mask[j] = 1;
        ++rounds;
    }
    free(add);
    return rounds;
}

/* Threshold modes. */
#define ORC_THR_EPS_NORMB 0   /* tau = eps ||b||_2 / sqrt(N)   (Sec. 2.3.1) */
#define ORC_THR_REL_MAX   1   /* tau = beta * max_i |r_i|      (relative variant) */
/* Expansion modes. */
#define ORC_EXP_NONE   0
#define ORC_EXP_DILATE 1      /* unconditional, `layers` graph layers */
#define ORC_EXP_PAPER  2      /* Alg 3, at most E_max rounds */

/* Residual-based local domain construction (Alg 3 / Eq. resi-local-domain-0),
 * with the relative-threshold and unconditional-dilation variants.  Writes
 * mask (0/1), r (initial residual) and tau; returns K. */
int32_t orc_mark_residual(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                          const double *b, const double *x0,
                          int32_t thr_mode, double param, int32_t exp_mode, int32_t rounds,
                          uint8_t *mask, double *r, double *tau_out, int32_t *rounds_out)
{
    orc_residual(n, rp, ci, av, b, x0, r);
    double tau;
    if (thr_mode == ORC_THR_EPS_NORMB) {
        tau = orc_tau_eps_normb(n, b, param);
    } else {
        double mx = 0.0;
        ORC_ROWS_MAX
        for (int32_t i = 0; i < n; ++i) if (fabs(r[i]) > mx) mx = fabs(r[i]);
        tau = param * mx;
    }
    ORC_ROWS
    for (int32_t i = 0; i < n; ++i) mask[i] = fabs(r[i]) > tau ? 1 : 0;
    int32_t done = 0;
    if (exp_mode == ORC_EXP_DILATE) {
        orc_dilate(n, rp, ci, av, mask, rounds);
        done = rounds;
    } else if (exp_mode == ORC_EXP_PAPER) {
        done = orc_expand_paper(n, rp, ci, av, r, x0, tau, mask, rounds, NULL);
    }
    if (tau_out) *tau_out = tau;
    if (rounds_out) *rounds_out = done;
    int32_t K = 0;
    for (int32_t i = 0; i < n; ++i) K += mask[i];
    return K;
}

/* Eq. grad (R4): g_i = sum over neighbours j of |x_i - x_j|. */
void orc_gradient(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                  const double *x, double *g)
{
    ORC_ROWS
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = ci[e];
            if (j == i || av[e] == 0.0) continue;
            s = s + fabs(x[i] - x[j]);
        }
        g[i] = s;
    }
}

/* Alg 2: gradient-based local domain, g_max initialised to 0, then
 * Omega = { i : g_i > alpha * g_max }, followed by `layers` dilation rounds
 * (0 = the paper's algorithm as printed).  Returns K. */
int32_t orc_mark_gradient(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                          const double *x0, double alpha, int32_t layers,
                          uint8_t *mask, double *g, double *gmax_out)
{
    orc_gradient(n, rp, ci, av, x0, g);
    double gmax = 0.0;
    for (int32_t i = 0; i < n; ++i) if (g[i] > gmax) gmax = g[i];
    double thr = alpha * gmax;
    for (int32_t i = 0; i < n; ++i) mask[i] = g[i] > thr ? 1 : 0;
    if (layers > 0) orc_dilate(n, rp, ci, av, mask, layers);
    if (gmax_out) *gmax_out = gmax;
    int32_t K = 0;
    for (int32_t i = 0; i < n; ++i) K += mask[i];
    return K;
}

/* ------------------------------------------------ extraction (Eq. loc-equ) */

/* Builds g2l/l2g (R8), the local block B = A[Omega, Omega] in local column
 * indices (values copied), rhs = b_B - E x_C^(0) (R2) and xL0 = x0[Omega].
 * Returns K; *nnzB_out receives nnz(B). */
int32_t orc_extract(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                    const uint8_t *mask, const double *b, const double *x0,
                    int32_t *g2l, int32_t *l2g, int32_t *brp, int32_t *bci, double *bav,
                    double *rhs, double *xL0, int32_t *nnzB_out)
{
    int32_t K = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (mask[i]) { g2l[i] = K; l2g[K] = i; ++K; }
        else g2l[i] = -1;
    }
    int32_t nz = 0;
    brp[0] = 0;
    for (int32_t l = 0; l < K; ++l) {
        int32_t i = l2g[l];
        double s = b[i];
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = ci[e];
            if (g2l[j] >= 0) { bci[nz] = g2l[j]; bav[nz] = av[e]; ++nz; }
            else s = fma(-av[e], x0[j], s);
        }
        rhs[l] = s;
        xL0[l] = x0[i];
        brp[l + 1] = nz;
    }
    if (nnzB_out) *nnzB_out = nz;
    return K;
}

/* Eq. sol-assemble: x~ = x0 with x~[l2g[l]] = xbar[l]. */
void orc_assemble(int32_t n, const double *x0, int32_t K, const int32_t *l2g,
                  const double *xbar, double *xt)
{
    memcpy(xt, x0, sizeof(double) * (size_t)n);
    for (int32_t l = 0; l < K; ++l) xt[l2g[l]] = xbar[l];
}

/* ----------------------------------------------------------- Krylov solve */

/* ||b - A x||_2 / ||b||_2 (Eq. rel-res-conv-criteria); 0 if b = 0 and r = 0. */
double orc_relres(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                  const double *b, const double *x)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    orc_residual(n, rp, ci, av, b, x, r);
    double rr = dot(n, r, r), bb = dot(n, b, b);
    free(r);
    if (bb == 0.0) return rr == 0.0 ? 0.0 : INFINITY;
    return sqrt(rr) / sqrt(bb);
}

/* Textbook Jacobi-preconditioned conjugate gradients (M = diag(A)), from the
 * initial iterate in x, stopping when ||r||_2^2 <= tol^2 ||b||_2^2 on the
 * recurrence residual; on that exit the true residual b - A x is recomputed
 * and, if it misses the tolerance, the iteration restarts from it (at most 3
 * restarts).  Returns 0, ORC_NOT_CONVERGED (x = last iterate) or
 * ORC_BREAKDOWN (p^T A p <= 0 or not finite). */
int32_t orc_pcg(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                const double *b, double *x, double tol, int32_t maxit,
                int32_t *iters_out, double *relres_out)
{
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double *r = (double *)malloc(sz), *z = (double *)malloc(sz), *p = (double *)malloc(sz);
    double *q = (double *)malloc(sz), *dinv = (double *)malloc(sz);
    int32_t status = ORC_NOT_CONVERGED, it = 0;
    ORC_ROWS
    for (int32_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) if (ci[e] == i) d = av[e];
        dinv[i] = 1.0 / d;
    }
    double bb = dot(n, b, b);
    double stop = (tol * tol) * bb;
    if (bb == 0.0) {                              /* A x = 0 has x = 0 */
        for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
        status = ORC_OK;
        goto done;
    }
    for (int restart = 0; restart <= 3; ++restart) {
        orc_residual(n, rp, ci, av, b, x, r);
        double rr = dot(n, r, r);
        if (rr <= stop) { status = ORC_OK; break; }
        ORC_ROWS
        for (int32_t i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
        double rz = dot(n, r, z);
        int converged = 0;
        while (it < maxit) {
            spmv(n, rp, ci, av, p, q);
            double pq = dot(n, p, q);
            if (!(pq > 0.0) || !isfinite(pq)) { status = ORC_BREAKDOWN; goto done; }
            double alpha = rz / pq;
            ORC_ROWS
            for (int32_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
            ++it;
            rr = dot(n, r, r);
            if (rr <= stop) { converged = 1; break; }
            ORC_ROWS
            for (int32_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
            double rz_new = dot(n, r, z);
            double beta = rz_new / rz;
            rz = rz_new;
            ORC_ROWS
            for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        if (!converged) { status = ORC_NOT_CONVERGED; break; }
        /* converged on the recurrence residual: confirm with the true one */
        orc_residual(n, rp, ci, av, b, x, r);
        if (dot(n, r, r) <= stop) { status = ORC_OK; break; }
    }
done:
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = orc_relres(n, rp, ci, av, b, x);
    free(r); free(z); free(p); free(q); free(dinv);
    return status;
}

/* ------------------------------------- Gauss-Seidel smoothing (Alg 1 step 7) */

/* One multicolour Gauss-Seidel sweep over A x = b (the whole system, Alg 1
 * step 7): for colour c = 0 .. ncol-1, for i ascending with colour[i] == c,
 *     s = b_i; for j ascending, j != i: s = fma(-a_ij, x_j, s); x_i = s / a_ii
 * using the newest x_j.  The caller's colouring gives no two neighbours the
 * same colour, so the sweep equals lexicographic Gauss-Seidel on the
 * colour-ordered system and does not depend on the order inside a colour
 * (red-black for the 5-point and 7-point stencils). */
void orc_gs_sweep(int32_t n, const int32_t *rp, const int32_t *ci, const double *av,
                  const double *b, double *x, const uint8_t *colour, int32_t ncol)
{
    for (int32_t c = 0; c < ncol; ++c)
        for (int32_t i = 0; i < n; ++i) {
            if (colour[i] != c) continue;
            double s = b[i], d = 0.0;
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
                if (ci[e] == i) d = av[e];
                else s = fma(-av[e], x[ci[e]], s);
            }
            x[i] = s / d;
        }
}

/* -------------------------------------------- Alg 1: local, then global */

#define ORC_MARK_RESIDUAL 0
#define ORC_MARK_GRADIENT 1

typedef struct {
    int32_t mark_mode;      /* ORC_MARK_RESIDUAL | ORC_MARK_GRADIENT */
    int32_t thr_mode;       /* residual marking: ORC_THR_* */
    double  thr_param;      /* eps (EPS_NORMB) or beta (REL_MAX) */
    int32_t exp_mode;       /* residual marking: ORC_EXP_* */
    int32_t exp_rounds;     /* layers (DILATE) or E_max (PAPER) */
    double  alpha;          /* gradient marking: alpha */
    int32_t grad_layers;    /* gradient marking: dilation layers */
    double  tol;            /* global tolerance eps of Eq. rel-res-conv-criteria */
    double  tol_local;      /* local solve tolerance, relative to ||rhs_L||_2 */
    int32_t maxit;
    int32_t gs_sweeps;      /* Gauss-Seidel sweeps of step 7 (0 = none) */
    int32_t gs_ncolours;    /* colours of the caller's colouring */
} orc_params;

typedef struct {
    int32_t K, nnzB, it_local, it_global, early_exit, status;
    double tau, relres_tilde, relres_final;
} orc_stats;

/* Alg 1: construct the local domain, extract and solve the subsystem from
 * x0[Omega], assemble x~, smooth it with gs_sweeps multicolour Gauss-Seidel
 * sweeps over the whole system (step 7; `colour` may be NULL when
 * gs_sweeps == 0), return it if it meets the criterion, else solve the whole
 * system from x~.  x holds x0 on entry and the solution on exit. */
int32_t orc_solve_local_then_global(int32_t n, const int32_t *rp, const int32_t *ci,
                                    const double *av, const double *b, double *x,
                                    const orc_params *prm, orc_stats *st, uint8_t *mask_out,
                                    const uint8_t *colour)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t nnz = rp[n];
    uint8_t *mask = (uint8_t *)malloc(nn);
    double *r = (double *)malloc(sizeof(double) * nn);
    int32_t *g2l = (int32_t *)malloc(sizeof(int32_t) * nn), *l2g = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *brp = (int32_t *)malloc(sizeof(int32_t) * (nn + 1));
    int32_t *bci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    double *bav = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double *rhs = (double *)malloc(sizeof(double) * nn), *xl = (double *)malloc(sizeof(double) * nn);
    double *xt = (double *)malloc(sizeof(double) * nn);
    memset(st, 0, sizeof(*st));

    if (prm->mark_mode == ORC_MARK_RESIDUAL) {
        orc_mark_residual(n, rp, ci, av, b, x, prm->thr_mode, prm->thr_param, prm->exp_mode,
                          prm->exp_rounds, mask, r, &st->tau, NULL);
    } else {
        orc_mark_gradient(n, rp, ci, av, x, prm->alpha, prm->grad_layers, mask, r, &st->tau);
    }
    int32_t nzB = 0;
    int32_t K = orc_extract(n, rp, ci, av, mask, b, x, g2l, l2g, brp, bci, bav, rhs, xl, &nzB);
    st->K = K;
    st->nnzB = nzB;
    int32_t status = ORC_OK;
    if (K > 0) {
        status = orc_pcg(K, brp, bci, bav, rhs, xl, prm->tol_local, prm->maxit, &st->it_local, NULL);
        if (status == ORC_BREAKDOWN) goto out;
    }
    orc_assemble(n, x, K, l2g, xl, xt);
    for (int32_t sw = 0; sw < prm->gs_sweeps; ++sw)
        orc_gs_sweep(n, rp, ci, av, b, xt, colour, prm->gs_ncolours);
    st->relres_tilde = orc_relres(n, rp, ci, av, b, xt);
    memcpy(x, xt, sizeof(double) * nn);
    if (st->relres_tilde <= prm->tol) {
        st->early_exit = 1;
        st->relres_final = st->relres_tilde;
        status = ORC_OK;
    } else {
        status = orc_pcg(n, rp, ci, av, b, x, prm->tol, prm->maxit, &st->it_global, &st->relres_final);
    }
out:
    st->status = status;
    if (mask_out) memcpy(mask_out, mask, (size_t)n);
    free(mask); free(r); free(g2l); free(l2g); free(brp); free(bci); free(bav);
    free(rhs); free(xl); free(xt);
    return status;
}

/* ----------------------------------------------------- adjoint gradient */

/* Gradient of L(x(k)) for the 2D 5-point operator of the generators
 * (T_f = 2 k_P k_N/(k_P+k_N), Dirichlet ghost 2 k_P on boundary faces), given
 * the state x and the adjoint lambda (A lambda = dL/dx, A symmetric):
 *   dL/dk_c = - sum_{faces f=(c,N)} 2 k_N^2/(k_c+k_N)^2 (lam_c - lam_N)(x_c - x_N)
 *             - sum_{boundary faces of c} 2 lam_c x_c.
 * Derived from dL/dk = -lambda^T (dA/dk) x. */
void orc_adjoint_grad_k_2d(int32_t nx, int32_t ny, const double *k, const double *x,
                           const double *lam, double *dk)
{
    for (int32_t y = 0; y < ny; ++y)
        for (int32_t xx = 0; xx < nx; ++xx) {
            int32_t c = xx + nx * y;
            double s = 0.0;
            int32_t nb[4] = { xx > 0 ? c - 1 : -1, xx < nx - 1 ? c + 1 : -1,
                              y > 0 ? c - nx : -1, y < ny - 1 ? c + nx : -1 };
            for (int f = 0; f < 4; ++f) {
                int32_t m = nb[f];
                if (m < 0) {
                    s += 2.0 * lam[c] * x[c];
                } else {
                    double den = k[c] + k[m];
                    double dT = 2.0 * k[m] * k[m] / (den * den);
                    s += dT * (lam[c] - lam[m]) * (x[c] - x[m]);
                }
            }
            dk[c] = -s;
        }
}

/* ------------------------------- nonlinear 2D heat conduction (Sec. 3.2) */

#define ORC_BC_DIRICHLET 0
#define ORC_BC_NEUMANN 1

/* Picard-linearised backward-Euler system of dT/dt = div(kappa(T) grad T) on
 * an nx x ny grid of cells of width h (Sec. 3.2, Eq. picard-equs), from the
 * cell conductivities kappa (evaluated at the previous Picard iterate) and
 * the previous time level Tn.  Sides in the order x-, x+, y-, y+; a Dirichlet
 * side holds T = bc_val through a ghost at half a cell (coefficient
 * 2 kappa_P/h^2, its value moved to b), a Neumann side has no flux.  With
 * c = 1/(h h) and faces visited W, E, S, N:
 *   T_f  = ((2 kappa_P) kappa_N / (kappa_P + kappa_N)) c    (interior face)
 *   g    = (2 kappa_P) c                                      (Dirichlet face)
 *   a_PP = 1/dt, then a_PP = a_PP + T_f or + g per face;  a_PN = -T_f
 *   b_P  = Tn_P (1/dt), then b_P = b_P + g bc_val per Dirichlet face.
 * CSR with ascending columns into rp[n+1], ci[5n], av[5n]; returns nnz. */
int32_t orc_heat2d_system(int32_t nx, int32_t ny, double h, double dt, const int32_t bc_type[4],
                          const double bc_val[4], const double *kappa, const double *Tn,
                          int32_t *rp, int32_t *ci, double *av, double *b)
{
    const double c = 1.0 / (h * h), inv_dt = 1.0 / dt;
    int32_t nz = 0;
    for (int32_t y = 0; y < ny; ++y)
        for (int32_t x = 0; x < nx; ++x) {
            const int32_t i = x + nx * y;
            const double kp = kappa[i];
            /* faces W, E, S, N: neighbour index or -1 with the side it lies on */
            const int32_t nb[4] = { x > 0 ? i - 1 : -1, x + 1 < nx ? i + 1 : -1,
                                    y > 0 ? i - nx : -1, y + 1 < ny ? i + nx : -1 };
            double tf[4];
            double d = inv_dt, bi = Tn[i] * inv_dt;
            for (int f = 0; f < 4; ++f) {
                tf[f] = 0.0;
                if (nb[f] >= 0) {
                    const double kn = kappa[nb[f]];
                    tf[f] = ((2.0 * kp) * kn / (kp + kn)) * c;
                    d = d + tf[f];
                } else if (bc_type[f] == ORC_BC_DIRICHLET) {
                    const double g = (2.0 * kp) * c;
                    d = d + g;
                    bi = bi + g * bc_val[f];
                }
            }
            rp[i] = nz;
            /* ascending columns: S (i-nx), W (i-1), P, E (i+1), N (i+nx) */
            if (nb[2] >= 0) { ci[nz] = nb[2]; av[nz++] = -tf[2]; }
            if (nb[0] >= 0) { ci[nz] = nb[0]; av[nz++] = -tf[0]; }
            ci[nz] = i; av[nz++] = d;
            if (nb[1] >= 0) { ci[nz] = nb[1]; av[nz++] = -tf[1]; }
            if (nb[3] >= 0) { ci[nz] = nb[3]; av[nz++] = -tf[3]; }
            b[i] = bi;
        }
    rp[nx * ny] = nz;
    return nz;
}

typedef struct {
    int32_t picard_its;   /* Picard iterations of the step */
    int32_t it_local;     /* CG iterations of all local solves */
    int32_t it_global;    /* CG iterations of all global solves */
    int32_t K_sum;        /* sum of |Omega_local| over the step's solves */
    int32_t early_exits;  /* solves whose x~ met the criterion */
    int32_t status;
    double  last_update;  /* ||T^{s+1} - T^s||_2 of the last iteration */
} orc_heat_stats;

/* One time step of the 2D heat problem by Picard iteration (Sec. 3.2, Alg. of
 * the 2-D heat solution): T holds T^{n+1,0} (normally T^n) on entry and
 * T^{n+1} on exit.  Each iteration s: kappa = T^p at T^{n+1,s}; assemble the
 * system; solve it from T^{n+1,s} by the global PCG (method 0) or by Alg 1
 * with prm's marking and smoothing (method 1; `colour` as for
 * orc_gs_sweep, NULL without smoothing); stop when ||T^{n+1,s+1} -
 * T^{n+1,s}||_2 < picard_tol or after max_picard iterations. */
int32_t orc_heat2d_step(int32_t nx, int32_t ny, double h, double dt, double p,
                        const int32_t bc_type[4], const double bc_val[4], const double *Tn, double *T,
                        int32_t method, const orc_params *prm, double picard_tol, int32_t max_picard,
                        orc_heat_stats *hs, const uint8_t *colour)
{
    const int32_t n = nx * ny;
    double *kappa = (double *)malloc(sizeof(double) * (size_t)n);
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *rp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(5 * n));
    double *av = (double *)malloc(sizeof(double) * (size_t)(5 * n));
    memset(hs, 0, sizeof(*hs));
    int32_t status = ORC_OK;
    for (int32_t s = 0; s < max_picard; ++s) {
        for (int32_t i = 0; i < n; ++i) kappa[i] = pow(T[i], p);
        orc_heat2d_system(nx, ny, h, dt, bc_type, bc_val, kappa, Tn, rp, ci, av, b);
        memcpy(x, T, sizeof(double) * (size_t)n);
        if (method == 0) {
            int32_t it = 0;
            status = orc_pcg(n, rp, ci, av, b, x, prm->tol, prm->maxit, &it, NULL);
            hs->it_global += it;
        } else {
            orc_stats st;
            status = orc_solve_local_then_global(n, rp, ci, av, b, x, prm, &st, NULL, colour);
            hs->it_local += st.it_local;
            hs->it_global += st.it_global;
            hs->K_sum += st.K;
            hs->early_exits += st.early_exit;
        }
        double d2 = 0.0;
        for (int32_t i = 0; i < n; ++i) d2 += (x[i] - T[i]) * (x[i] - T[i]);
        memcpy(T, x, sizeof(double) * (size_t)n);
        hs->picard_its = s + 1;
        hs->last_update = sqrt(d2);
        if (status != ORC_OK || hs->last_update < picard_tol) break;
    }
    hs->status = status;
    free(kappa); free(b); free(x); free(rp); free(ci); free(av);
    return status;
}

/* Threads the parallel loops use: omp_get_max_threads() in the OpenMP build,
 * 1 in the serial oracle. */
int32_t orc_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
