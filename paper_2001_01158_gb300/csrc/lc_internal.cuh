// lc_internal.cuh -- host-side declarations of the lc library: workspaces,
// launch parameters and the launchers of every kernel file.  Device helpers
// and descriptors live in lc_device.cuh.
//
// Nothing here is part of the public ABI (include/lc_api.h).
#pragma once

#include "lc_device.cuh"

namespace lc {

// ---------------------------------------------------------------- host side

struct Launch {
    cudaStream_t stream;
};

// Accounting of kernel launches (lc_kernel_launch_count).
void note_launches(int n);

// Batched Alg 1 (lc_batched.cu): many independent 2D systems in one launch
struct BatchView {
    int nsys;
    const int32_t *nx, *ny;
    const int64_t *off;        // cell offset of each system
    const int32_t *order;      // processing order (largest first)
    const double *D, *Tx, *Ty; // FP64 operator (caller's, concatenated)
    const float *D32, *Tx32, *Ty32, *dinv32;   // FP32 copies (library's)
    const double *b;
    double *x;
    // workspace, concatenated like the cells (capacities: cells, 5 x cells for B)
    double *r;                 // FP64 residual
    uint8_t *m0, *m1;          // masks
    int32_t *g2l, *l2g, *rowptr;   // rowptr: cells + nsys (offset off[s] + s)
    int32_t *col;              // 5 x cells (offset 5 off[s])
    double *val;
    float *val32;
    double *rhs, *xl;
    float *dl32;               // 1/diag(B) in FP32
    float *r32, *z32, *p32, *q32, *d32;
    int32_t *next;             // work-queue counters: [0] systems solved by clusters, [1] by single CTAs
    int nbig;                  // the first nbig systems of `order` are solved by clusters (0 without clusters)
    int32_t *stat_i;           // [nsys][8]: status, K, nnzB, it_local, it_global, outer_local, outer_global, early
    double *stat_d;            // [nsys][4]: tau, relres_tilde, relres_final, bnorm
};

struct BatchParams {
    double beta;
    int layers;
    double tol, tol_local, inner_tol;
    int max_outer, max_inner;
};

struct BatchLaunch {
    BatchView v;
    BatchParams p;
    int block;       // 256, 512 or 1024
    int ctas_per_sm; // 0 = as many as fit
    int cluster;     // CTAs per thread-block cluster: 1 (none), 2, 4, 8 or 16
    int64_t big_cells;  // with clusters: systems of at least this many cells are solved by a whole cluster
};

cudaError_t launch_batched(const void *launch_desc, int sms, cudaStream_t s);
cudaError_t launch_batch_f32(int64_t n, const double *D, const double *Tx, const double *Ty, float *D32, float *Tx32,
                             float *Ty32, float *dinv32, cudaStream_t s);
int batched_occupancy(int block);

// Operator assembly and adjoint gradient (lc_adjoint.cu)
cudaError_t launch_assemble_2d(int nx, int ny, const double *k, double dt, double *D, double *Tx, double *Ty,
                               cudaStream_t s);
cudaError_t launch_adjoint_grad_k_2d(int nx, int ny, const double *k, const double *x, const double *lam, double *dk,
                                     cudaStream_t s);

// Launchers (one translation unit each).  All return cudaError_t of the
// last launch; argument validation happens in lc_api.cu.
cudaError_t launch_residual_stencil(const Stencil &op, const double *b, const double *x, double *r,
                                    int want_tree, double *tree_partials, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_residual_csr(const Csr &op, const double *b, const double *x, double *r,
                                int want_tree, double *tree_partials, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_tree_finish(double *partials, double *scratch, int64_t nchunks, int64_t n, double eps,
                               Ctrl *ctrl, double *tau_out, cudaStream_t s);
cudaError_t launch_tau_relmax(double beta, Ctrl *ctrl, double *tau_out, cudaStream_t s);
cudaError_t launch_threshold_dilate_stencil(const Stencil &op, const double *v, int layers, uint8_t *mask,
                                            Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_dilate_stencil_pass(const Stencil &op, int layers, const uint8_t *in, uint8_t *out, cudaStream_t s);
// Threshold and `layers` graph layers through bit-packed rows (any layer
// count): bits_a, bits_b hold ny nz bits_words(op) words each.
int bits_words(const Stencil &op);
cudaError_t launch_threshold_dilate_bits(const Stencil &op, const double *v, int layers, uint8_t *mask,
                                         uint32_t *bits_a, uint32_t *bits_b, Ctrl *ctrl, cudaStream_t s);
inline int max_layers_per_pass(int dim) { return dim == 3 ? 2 : 4; }
cudaError_t launch_threshold_csr(int32_t n, const double *v, uint8_t *mask, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_dilate_csr(const Csr &op, const uint8_t *in, uint8_t *out, cudaStream_t s);
cudaError_t launch_expand_paper_stencil(const Stencil &op, const double *r, const double *x0, int round,
                                        const uint8_t *in, uint8_t *out, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_expand_paper_csr(const Csr &op, const double *r, const double *x0, int round,
                                    const uint8_t *in, uint8_t *out, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_gradient_stencil(const Stencil &op, const double *x, double *g, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_gradient_csr(const Csr &op, const double *x, double *g, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_gmax_threshold(double alpha, Ctrl *ctrl, double *gmax_out, cudaStream_t s);
cudaError_t launch_count_mask(int64_t n, const uint8_t *mask, Ctrl *ctrl, int32_t *K_out, cudaStream_t s);

// Extraction (lc_extract.cu)
struct ExtractWork {
    unsigned long long *blk;   // per-block packed (cells, entries) totals, capacity >= nblocks + 1
    int64_t nblocks_cap;
};
cudaError_t launch_extract_stencil(const Stencil &op, const uint8_t *mask, const double *b, const double *x0,
                                   const lc_subsys &out, ExtractWork &w, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_extract_csr(const Csr &op, const uint8_t *mask, const double *b, const double *x0,
                               const lc_subsys &out, ExtractWork &w, Ctrl *ctrl, cudaStream_t s);
cudaError_t launch_assemble(const int32_t *K_dev, const int32_t *l2g, const double *xbar, double *x, int64_t cap,
                            cudaStream_t s);

// Gauss-Seidel smoothing, Alg 1 step 7 (lc_smooth.cu): `sweeps` multicolour
// sweeps in place -- red-black for stencils, the caller's colouring for CSR
cudaError_t launch_gs_stencil(const Stencil &s, const double *b, double *x, int sweeps, cudaStream_t st);
cudaError_t launch_gs_csr(const Csr &cs, const uint8_t *colour, int ncol, const double *b, double *x, int sweeps,
                          cudaStream_t st);
cudaError_t launch_check_colouring(const Csr &cs, const uint8_t *colour, int ncol, int *bad, cudaStream_t st);

// Nonlinear 2D heat problem, Sec. 3.2 (lc_heat.cu)
struct HeatBc {
    int type[4];     // sides x-, x+, y-, y+: LC_BC_DIRICHLET | LC_BC_NEUMANN
    double val[4];   // Dirichlet values
};
cudaError_t launch_heat_kappa(int64_t n, const double *T, double p, double *kappa, cudaStream_t s);
cudaError_t launch_heat_assemble(int nx, int ny, double h, double dt, const HeatBc &bc, const double *kappa,
                                 const double *Tn, double *D, double *Tx, double *Ty, double *b, cudaStream_t s);
// *out = sum (x - y)^2 (deterministic); part: >= 608 doubles of scratch
cudaError_t launch_diff2(int64_t n, const double *x, const double *y, double *part, double *out, cudaStream_t s);

// Reproducible dot product (lc_dot.cu): *out = sum x_i y_i, products summed
// exactly in fixed point; scratch >= 2 + 2 * 608 64-bit words
cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *out, double *scratch, cudaStream_t s);

// Self-test of the bounded grid barrier (lc_selftest.cu): a barrier that
// cannot complete; *passed counts blocks that wrongly got through
cudaError_t launch_barrier_timeout_selftest(Ctrl *ctrl, int *passed, int blocks, long long limit_cycles,
                                            cudaStream_t s);

// Krylov (lc_pcg_impl.cuh kernels; lc_pcg.cu, lc_pcg_mixed.cu, lc_pcg3d.cu, lc_pcgcsr.cu launches)
struct PcgWork {
    double *r, *z, *p0, *p1, *q;     // capacity n
    double *e0, *e1;                 // capacity n (single-reduction CSR solve)
    double *dinv;                    // CSR: per-row 1/a_ii (capacity n)
    double *partials;                // kMaxGrid * 8
    float *r32, *z32, *p032, *p132, *q32, *x32, *dinv32;   // mixed precision (capacity n)
    float *val32;                    // mixed precision, CSR: FP32 values (capacity nnz)
    double *xh;                      // pipelined local solve: the scaled iterate (capacity n)
    double *ahat;                    // pipelined local solve: D^-1/2 B D^-1/2 values (capacity nnz)
};
struct PcgArgs {
    const double *b;
    double *x;
    double tol;
    int32_t maxit;
    int32_t max_restarts;
    int32_t minblocks;    // register budget of the structured-grid kernel (tuning)
    int32_t precision;    // LC_PREC_FP64 | LC_PREC_MIXED
    double inner_tol;     // mixed: reduction asked of each FP32 inner solve
    int32_t max_outer;    // mixed: refinement sweeps
    int32_t scaled;       // FP64 2D: iterate on the symmetrically scaled system (tuning)
    int32_t wide;         // FP64 2D scaled: four cells per lane (tuning)
    int32_t big;          // 2D solves: one block of 768 threads per SM (tuning)
    int32_t pairdot;      // FP64 2D scaled wide: dot products and block sums on FP32 pairs (tuning)
    int32_t lazyx;        // FP64 2D scaled wide pair: x += alpha p in the next phase A (tuning)
    int32_t store_p;      // global CSR systems: p stored once per row before the product (tuning)
};
cudaError_t launch_pcg_stencil(const Stencil &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                               cudaStream_t s);
// the parts of launch_pcg_stencil in their own translation units
cudaError_t launch_pcg_stencil3d(const Stencil &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                                 cudaStream_t s);
cudaError_t launch_ir_stencil2d(const Stencil &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                                cudaStream_t s);
// after_cluster: launched right after launch_pcg_csr_cluster on the same
// ctrl -- no reset of ctrl, and the kernel returns at once if ctrl->done
cudaError_t launch_pcg_csr(const Csr &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                           cudaStream_t s, bool after_cluster = false);
// FP64 Jacobi-PCG of a CSR system with one grid reduction per iteration
// (lc_pcg1.cu); after_cluster as for launch_pcg_csr
cudaError_t launch_pcg_csr_single(const Csr &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                                  cudaStream_t s, bool after_cluster);
// Pipelined Jacobi-PCG (one grid barrier per iteration, the sums read while
// the product runs) for the extracted local subsystem (lc_pcgpipe.cu); with
// a.precision LC_PREC_MIXED its FP32 form inside FP64 iterative refinement.
cudaError_t launch_pcg_csr_pipelined(const Csr &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                                     cudaStream_t s, bool after_cluster);
// FP64 Jacobi-PCG of a CSR system on one thread-block cluster (lc_cluster.cu),
// when it has at most max_rows rows and they fit the cluster's shared memory
// (cluster_local_rows(); 0 if the device cannot run the cluster); sets
// ctrl->done
int cluster_local_rows();
cudaError_t launch_pcg_csr_cluster(const Csr &op, const PcgArgs &a, int max_rows, int threads, int ctas, Ctrl *ctrl,
                                   cudaStream_t s);
cudaError_t launch_dinv_stencil(int64_t n, const double *D, double *dinv, float *D32, const double *Tx,
                                const double *Ty, const double *Tz, float *Tx32, float *Ty32, float *Tz32,
                                float *dinv32, cudaStream_t s);
cudaError_t launch_check_stencil(const Stencil &op, int *bad, cudaStream_t s);
// Symmetric scaling S = D^-1/2 of a stencil operator (2D or 3D): sc = S,
// sq = S^-1, T^ = T S_P S_N per face (0 on the last column/row/plane; Tzh only
// in 3D), dn32 and dexp as described in Stencil, FP32 copies of the scaled
// faces and of sq; two launches
cudaError_t launch_scaling(const Stencil &st, double *sc, double *sq, double *Txh, double *Tyh, double *Tzh,
                           float *dn32, int *dexp, float *Txh32, float *Tyh32, float *Tzh32, float *sq32,
                           cudaStream_t s);
cudaError_t launch_check_csr(int32_t n, const int32_t *rp, const int32_t *ci, const double *av, int *bad,
                             cudaStream_t s);

}  // namespace lc
