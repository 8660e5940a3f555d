// lc_extract.cu -- the local subsystem B x_B = b_B - E x_C^(0) (Eq. loc-equ)
// and the assembly x~ = Q [xbar_B; x_C^(0)] (Eq. sol-assemble).
//
// One exclusive scan over the cells produces both index maps and the row
// pointers of B: every local cell contributes the packed pair
//     (1, 1 + number of local neighbours)   as  low | high << 32
// so the prefix of the low halves is the local index (ascending global
// order, a symmetric permutation of the paper's Q) and the prefix of the
// high halves is the row start in B.  Then a gather pass copies the local
// entries of each local row (values bit for bit, columns through g2l) and
// forms rhs_l = b_i; rhs_l = fma(-a_ij, x0_j, rhs_l) over the non-local j
// ascending -- the canonical order of include/lc_api.h.
//
// Passes: count (1 B/cell mask + neighbour masks) -> scan of block totals
// (one block) -> write g2l / l2g / rowptr -> gather K rows (~5-7 entries).
#include "lc_internal.cuh"

namespace lc {

namespace {

constexpr int kXThreads = 256;
constexpr int kXCells = 4;                     // consecutive cells per thread
constexpr int kXChunk = kXThreads * kXCells;   // cells per block

template <int DIM>
__device__ __forceinline__ unsigned count_local_nbrs(const Stencil &op, const uint8_t *__restrict__ mask, int64_t i) {
    const int64_t sxy = (int64_t)op.nx * op.ny;
    const unsigned ux = (unsigned)(i % op.nx);
    const unsigned uy = (unsigned)((i / op.nx) % op.ny);
    unsigned c = 0;
    if (DIM == 3) {
        const unsigned uz = (unsigned)(i / sxy);
        if (uz > 0) c += mask[i - sxy];
        if (uz + 1 < (unsigned)op.nz) c += mask[i + sxy];
    }
    if (uy > 0) c += mask[i - op.nx];
    if (ux > 0) c += mask[i - 1];
    if (ux + 1 < (unsigned)op.nx) c += mask[i + 1];
    if (uy + 1 < (unsigned)op.ny) c += mask[i + op.nx];
    return c;
}

__device__ __forceinline__ unsigned count_local_csr(const Csr &op, const uint8_t *__restrict__ mask, int64_t i) {
    unsigned c = 0;
    const int32_t e1 = op.rp[i + 1];
    for (int32_t e = op.rp[i]; e < e1; ++e) c += mask[LC_IDX(op.ci[e], op.n)];
    return c;   // includes the diagonal (mask[i] == 1 for a local row)
}

template <class OP, int DIM>
__device__ __forceinline__ unsigned long long cell_pair(const OP &op, const uint8_t *__restrict__ mask, int64_t i);

template <>
__device__ __forceinline__ unsigned long long cell_pair<Stencil, 2>(const Stencil &op, const uint8_t *__restrict__ mask,
                                                                    int64_t i) {
    if (i >= op.n || !mask[i]) return 0ull;
    return 1ull | ((unsigned long long)(1u + count_local_nbrs<2>(op, mask, i)) << 32);
}
template <>
__device__ __forceinline__ unsigned long long cell_pair<Stencil, 3>(const Stencil &op, const uint8_t *__restrict__ mask,
                                                                    int64_t i) {
    if (i >= op.n || !mask[i]) return 0ull;
    return 1ull | ((unsigned long long)(1u + count_local_nbrs<3>(op, mask, i)) << 32);
}
template <>
__device__ __forceinline__ unsigned long long cell_pair<Csr, 0>(const Csr &op, const uint8_t *__restrict__ mask,
                                                                int64_t i) {
    if (i >= op.n || !mask[i]) return 0ull;
    return 1ull | ((unsigned long long)count_local_csr(op, mask, i) << 32);
}

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long w = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += w;
    }
    return v;
}

// Exclusive block scan of one value per thread; returns the exclusive prefix
// and writes the block total to *total (all threads).
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long *sm,
                                                              unsigned long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    unsigned long long inc = warp_incl_scan(v);
    __syncthreads();
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? sm[lane] : 0ull;
        w = warp_incl_scan(w);
        if (lane < nw) sm[lane] = w;
    }
    __syncthreads();
    const unsigned long long before = warp > 0 ? sm[warp - 1] : 0ull;
    *total = sm[nw - 1];
    return before + inc - v;
}

template <class OP, int DIM>
__global__ void __launch_bounds__(kXThreads) count_kernel(OP op, int64_t n, const uint8_t *__restrict__ mask,
                                                          unsigned long long *__restrict__ blk) {
    __shared__ unsigned long long sm[32];
    const int64_t base = (int64_t)blockIdx.x * kXChunk + (int64_t)threadIdx.x * kXCells;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kXCells; ++k) s += cell_pair<OP, DIM>(op, mask, base + k);
    unsigned long long tot;
    block_excl_scan(s, sm, &tot);
    if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

// Exclusive scan of the block totals in place (single block of 1024
// threads, each thread a contiguous segment); writes K, nnz(B) and
// rowptr[K] = nnz(B).
__global__ void __launch_bounds__(1024) scan_blocks_kernel(unsigned long long *__restrict__ blk, int64_t nb,
                                                           int32_t *rowptr, int32_t *K_out, int32_t *nnz_out,
                                                           Ctrl *ctrl) {
    __shared__ unsigned long long sm[32];
    const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = threadIdx.x * per;
    const int64_t b1 = b0 + per < nb ? b0 + per : nb;
    unsigned long long s = 0;
    for (int64_t b = b0; b < b1; ++b) s += blk[b];
    unsigned long long tot;
    unsigned long long off = block_excl_scan(s, sm, &tot);
    for (int64_t b = b0; b < b1; ++b) {
        const unsigned long long v = blk[b];
        blk[b] = off;
        off += v;
    }
    if (threadIdx.x == 0) {
        const int32_t K = (int32_t)(tot & 0xffffffffull);
        const int32_t nz = (int32_t)(tot >> 32);
        rowptr[K] = nz;
        *K_out = K;
        *nnz_out = nz;
        ctrl->K = K;
        ctrl->nnzB = nz;
    }
}

template <class OP, int DIM>
__global__ void __launch_bounds__(kXThreads) write_maps_kernel(OP op, int64_t n, const uint8_t *__restrict__ mask,
                                                               const unsigned long long *__restrict__ blk,
                                                               int32_t *__restrict__ g2l, int32_t *__restrict__ l2g,
                                                               int32_t *__restrict__ rowptr) {
    __shared__ unsigned long long sm[32];
    const int64_t base = (int64_t)blockIdx.x * kXChunk + (int64_t)threadIdx.x * kXCells;
    unsigned long long v[kXCells];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kXCells; ++k) { v[k] = cell_pair<OP, DIM>(op, mask, base + k); s += v[k]; }
    unsigned long long tot;
    unsigned long long off = block_excl_scan(s, sm, &tot) + blk[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kXCells; ++k) {
        const int64_t i = base + k;
        if (i < n) {
            if (v[k]) {
                const int32_t l = (int32_t)(off & 0xffffffffull);
                g2l[i] = l;
                l2g[LC_IDX(l, n)] = (int32_t)i;
                rowptr[l] = (int32_t)(off >> 32);
            } else {
                g2l[i] = -1;
            }
        }
        off += v[k];
    }
}

// Gather of one local row l (global i) of a stencil operator.
template <int DIM>
__global__ void __launch_bounds__(256) gather_stencil_kernel(Stencil op, const int32_t *__restrict__ Kp,
                                                             const int32_t *__restrict__ l2g,
                                                             const int32_t *__restrict__ g2l,
                                                             const int32_t *__restrict__ rowptr,
                                                             const double *__restrict__ b,
                                                             const double *__restrict__ x0, int32_t *__restrict__ col,
                                                             double *__restrict__ val, double *__restrict__ rhs,
                                                             double *__restrict__ xL0) {
    const int32_t K = *Kp;
    const int64_t sxy = (int64_t)op.nx * op.ny;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < K; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = LC_IDX(l2g[l], op.n);
        const unsigned ux = (unsigned)(i % op.nx);
        const unsigned uy = (unsigned)((i / op.nx) % op.ny);
        const unsigned uz = DIM == 3 ? (unsigned)(i / sxy) : 0u;
        int32_t e = rowptr[l];
        double s = b[i];
        // neighbour j with coefficient -T (T > 0): local -> entry, else rhs
        auto visit = [&](int64_t j, double T) {
            const int32_t gj = g2l[j];
            if (gj >= 0) { col[e] = LC_IDX(gj, K); val[e] = -T; ++e; }
            else s = __fma_rn(T, x0[j], s);
        };
        if (DIM == 3 && uz > 0) visit(i - sxy, op.Tz[i - sxy]);
        if (uy > 0) visit(i - op.nx, op.Ty[i - op.nx]);
        if (ux > 0) visit(i - 1, op.Tx[i - 1]);
        col[e] = (int32_t)l; val[e] = op.D[i]; ++e;
        if (ux + 1 < (unsigned)op.nx) visit(i + 1, op.Tx[i]);
        if (uy + 1 < (unsigned)op.ny) visit(i + op.nx, op.Ty[i]);
        if (DIM == 3 && uz + 1 < (unsigned)op.nz) visit(i + sxy, op.Tz[i]);
        rhs[l] = s;
        xL0[l] = x0[i];
    }
}

__global__ void __launch_bounds__(256) gather_csr_kernel(Csr op, const int32_t *__restrict__ Kp,
                                                         const int32_t *__restrict__ l2g,
                                                         const int32_t *__restrict__ g2l,
                                                         const int32_t *__restrict__ rowptr,
                                                         const double *__restrict__ b, const double *__restrict__ x0,
                                                         int32_t *__restrict__ col, double *__restrict__ val,
                                                         double *__restrict__ rhs, double *__restrict__ xL0) {
    const int32_t K = *Kp;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < K; l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = LC_IDX(l2g[l], op.n);
        int32_t e = rowptr[l];
        double s = b[i];
        const int32_t e1 = op.rp[i + 1];
        for (int32_t a = op.rp[i]; a < e1; ++a) {
            const int32_t j = LC_IDX(op.ci[a], op.n);
            const int32_t gj = g2l[j];
            if (gj >= 0) { col[e] = LC_IDX(gj, K); val[e] = op.av[a]; ++e; }
            else s = __fma_rn(-op.av[a], x0[j], s);
        }
        rhs[l] = s;
        xL0[l] = x0[i];
    }
}

__global__ void assemble_kernel(const int32_t *__restrict__ Kp, const int32_t *__restrict__ l2g,
                                const double *__restrict__ xbar, double *__restrict__ x, int64_t n) {
    const int32_t K = *Kp;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < K; l += (int64_t)gridDim.x * blockDim.x)
        x[LC_IDX(l2g[l], n)] = xbar[l];
}

inline unsigned flat_grid(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

template <class OP, int DIM>
cudaError_t run_maps(const OP &op, int64_t n, const uint8_t *mask, const lc_subsys &out, ExtractWork &w, Ctrl *ctrl,
                     cudaStream_t s) {
    const int64_t nb = (n + kXChunk - 1) / kXChunk;
    if (nb + 1 > w.nblocks_cap) return cudaErrorInvalidValue;
    count_kernel<OP, DIM><<<(unsigned)nb, kXThreads, 0, s>>>(op, n, mask, w.blk);
    note_launches(1);
    scan_blocks_kernel<<<1, 1024, 0, s>>>(w.blk, nb, out.rowptr, out.K, out.nnz, ctrl);
    note_launches(1);
    write_maps_kernel<OP, DIM><<<(unsigned)nb, kXThreads, 0, s>>>(op, n, mask, w.blk, out.g2l, out.l2g, out.rowptr);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_extract_stencil(const Stencil &op, const uint8_t *mask, const double *b, const double *x0,
                                   const lc_subsys &out, ExtractWork &w, Ctrl *ctrl, cudaStream_t s) {
    cudaError_t e = op.dim == 3 ? run_maps<Stencil, 3>(op, op.n, mask, out, w, ctrl, s)
                                : run_maps<Stencil, 2>(op, op.n, mask, out, w, ctrl, s);
    if (e != cudaSuccess) return e;
    if (op.dim == 3)
        gather_stencil_kernel<3><<<flat_grid(op.n), 256, 0, s>>>(op, out.K, out.l2g, out.g2l, out.rowptr, b, x0, out.col,
                                                                  out.val, out.rhs, out.xL0);
    else
        gather_stencil_kernel<2><<<flat_grid(op.n), 256, 0, s>>>(op, out.K, out.l2g, out.g2l, out.rowptr, b, x0, out.col,
                                                                  out.val, out.rhs, out.xL0);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_extract_csr(const Csr &op, const uint8_t *mask, const double *b, const double *x0,
                               const lc_subsys &out, ExtractWork &w, Ctrl *ctrl, cudaStream_t s) {
    cudaError_t e = run_maps<Csr, 0>(op, op.n, mask, out, w, ctrl, s);
    if (e != cudaSuccess) return e;
    gather_csr_kernel<<<flat_grid(op.n), 256, 0, s>>>(op, out.K, out.l2g, out.g2l, out.rowptr, b, x0, out.col, out.val,
                                                      out.rhs, out.xL0);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_assemble(const int32_t *K_dev, const int32_t *l2g, const double *xbar, double *x, int64_t cap,
                            cudaStream_t s) {
    assemble_kernel<<<flat_grid(cap), 256, 0, s>>>(K_dev, l2g, xbar, x, cap);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace lc
