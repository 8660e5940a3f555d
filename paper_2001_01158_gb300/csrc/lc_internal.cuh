// lc_internal.cuh -- shared device helpers and descriptors of the lc library.
//
// Nothing here is part of the public ABI (include/lc_api.h).  All kernels
// are written for sm_103a: 32-wide warps, 152 SMs, FP64 at roughly 1/12 of
// a DP op per HBM byte -- so every bit-exact kernel spends exactly the FP64
// operations its canonical order names and does abs/max/compare on integer
// bit patterns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lc_api.h"

namespace lc {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTreeChunk = 1024;                       // canonical sum-of-squares chunk
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;
constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr int kMaxExpRounds = 64;
constexpr int kMaxGrid = 4096;                          // persistent-kernel blocks (partials capacity)

// ---------------------------------------------------------------- descriptors

// Structured operator: the diagonal D and face conductances T (off-diagonal
// -T); dinv = 1/D precomputed at creation.  Cell i = x + nx*(y + ny*z).
struct Stencil {
    int dim;
    int nx, ny, nz;
    int64_t n;
    const double *D, *Tx, *Ty, *Tz;
    const double *dinv;
    // FP32 copies for the mixed-precision inner solve (fl32 of the above)
    const float *D32, *Tx32, *Ty32, *Tz32, *dinv32;
    // symmetric Jacobi scaling S = D^-1/2 (FP64 solve): S^-1 = D^1/2 and the
    // scaled face conductances T_f / sqrt(D_P D_N) of S A S (unit diagonal);
    // dn32 = fl32(D 2^-2h), h = floor(e/2), e the largest binary exponent of
    // D, stored biased (+1023) in *dexp
    const double *sc, *sq, *Txh, *Tyh;
    const float *dn32;
    const int *dexp;
};

// CSR operator; rows ascending, diagonal present.  `n_dev`, if not null,
// holds the row count on the device (used for extracted subsystems whose
// size is only known on the device); otherwise `n` is the count.
struct Csr {
    int32_t n;
    const int32_t *n_dev;
    const int32_t *rp, *ci;
    const double *av;
    const float *av32;
};

// Device-resident control block of one operator (one per lc_op).
struct Ctrl {
    // grid barrier
    unsigned long long bar_count;   // arrivals since the launch started (zeroed before it)
    int32_t status;                 // first error a kernel raised (LC_OK if none)
    int32_t done;                   // local solve: 1 if the cluster kernel solved the system
    // marking
    unsigned long long maxabs_bits; // max |r| (or max g) as bits, NaN excluded
    double tau;
    int32_t K;
    int32_t nnzB;
    int32_t added[kMaxExpRounds];   // Alg 3: K0 of each round
    // Krylov
    int32_t iters;
    int32_t restarts;
    int32_t converged;              // 1 ok, 0 not converged, -1 breakdown
    int32_t early;                  // converged at set-up (x0 already met the criterion)
    double relres0;                 // relative residual of the starting iterate
    double relres;                  // final relative residual (true residual)
    double bnorm2;                  // ||b||^2
    // mixed-precision refinement
    int32_t outer;
    int32_t pad1;
    double scale;                   // ||r|| of the current outer residual
};

// ---------------------------------------------------------------- bit helpers

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & kAbsMask;
}
// |v| > t exactly as IEEE compares it, given tbits = abs_bits(t), t >= 0 or
// NaN: a NaN |v| never exceeds, nothing exceeds a NaN t or +inf.
__device__ __forceinline__ bool abs_gt(double v, unsigned long long tbits) {
    unsigned long long a = abs_bits(v);
    return a > tbits && a <= kInfBits && tbits <= kInfBits;
}
// bits of |v| for a max that ignores NaN (as `if (|v| > m) m = |v|` does)
__device__ __forceinline__ unsigned long long maxable_bits(double v) {
    unsigned long long a = abs_bits(v);
    return a <= kInfBits ? a : 0ull;
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_down_sync(kFull, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ int warp_isum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// Deterministic block sum of NV values per thread (result valid in thread 0).
// `sm` needs NV * 32 doubles.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[k * 32 + warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            T t = lane < nw ? sm[k * 32 + lane] : T(0);
            v[k] = warp_sum(t);
        }
    }
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sm[lane] : 0ull;
        v = warp_max(v);
    }
    return v;
}

__device__ __forceinline__ int block_isum(int v, int *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_isum(v);
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sm[lane] : 0;
        v = warp_isum(v);
    }
    return v;
}

// ---------------------------------------------------------------- grid barrier

// Spin limit of every grid-wide wait: ~2 s at 2 GHz, after which the block
// records LC_ERR_TIMEOUT in ctrl->status and returns false; the other blocks
// stop at their own next wait, bounded the same way, and kernels exit.  Co-residency of all
// blocks is guaranteed by the cooperative launch.
constexpr long long kBarrierTimeoutCycles = 4000000000ll;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Counting barrier: arrival k of a block (k = 0, 1, ...) takes the counter
// from somewhere in [k n, (k+1) n) and the barrier opens when it reaches
// (k+1) n, so the target follows from the value the arrival returns: one
// atomic per block and arrival, no generation word, no reset between
// barriers.  A block never sees the counter past its own target before it
// arrives (no block passes barrier k before all arrived).
__device__ __forceinline__ bool grid_sync(Ctrl *ctrl, unsigned int nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();   // the block's writes (ordered by the barrier above) before the arrival
        const unsigned long long old = atomicAdd(&ctrl->bar_count, 1ull);
        const unsigned long long target = (old / nblocks + 1) * nblocks;
        int ok = 1;
        if (old + 1 < target) {
            const long long t0 = clock64();
            while (ld_acquire_u64(&ctrl->bar_count) < target) {
                if (clock64() - t0 > kBarrierTimeoutCycles) { ok = 0; break; }
            }
        }
        __threadfence();
        if (!ok) atomicCAS(&ctrl->status, LC_OK, LC_ERR_TIMEOUT);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Loads of data that other blocks of the same (persistent) kernel write:
// bypass L1, which is not coherent across SMs.
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }


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
    int32_t *next;             // work-queue counter
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

// Krylov (lc_pcg.cu)
struct PcgWork {
    double *r, *z, *p0, *p1, *q;     // capacity n
    double *dinv;                    // CSR: per-row 1/a_ii (capacity n)
    double *partials;                // kMaxGrid * 8
    float *r32, *z32, *p032, *p132, *q32, *x32, *dinv32;   // mixed precision (capacity n)
    float *val32;                    // mixed precision, CSR: FP32 values (capacity nnz)
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
};
cudaError_t launch_pcg_stencil(const Stencil &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                               cudaStream_t s);
// after_cluster: launched right after launch_pcg_csr_cluster on the same
// ctrl -- no reset of ctrl, and the kernel returns at once if ctrl->done
cudaError_t launch_pcg_csr(const Csr &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                           cudaStream_t s, bool after_cluster = false);
// FP64 Jacobi-PCG of a CSR system on one thread-block cluster (lc_cluster.cu),
// when it has at most max_rows rows and they fit the cluster's shared memory
// (cluster_local_rows(); 0 if the device cannot run the cluster); sets
// ctrl->done
int cluster_local_rows();
cudaError_t launch_pcg_csr_cluster(const Csr &op, const PcgArgs &a, int max_rows, int threads, Ctrl *ctrl,
                                   cudaStream_t s);
cudaError_t launch_dinv_stencil(int64_t n, const double *D, double *dinv, float *D32, const double *Tx,
                                const double *Ty, const double *Tz, float *Tx32, float *Ty32, float *Tz32,
                                float *dinv32, cudaStream_t s);
cudaError_t launch_check_stencil(const Stencil &op, int *bad, cudaStream_t s);
// 2D: sc = D^-1/2, sq = D^1/2, Txh/Tyh = T / sqrt(D_P D_N) (0 on the last
// column/row), dn32 and dexp as described in Stencil; two launches
cudaError_t launch_scaling_2d(const Stencil &st, double *sc, double *sq, double *Txh, double *Tyh, float *dn32,
                              int *dexp, cudaStream_t s);
cudaError_t launch_check_csr(int32_t n, const int32_t *rp, const int32_t *ci, const double *av, int *bad,
                             cudaStream_t s);

}  // namespace lc
