// lc_mark.cu -- construction of the local domain on the GPU.
//
//   residual  r0 = b - A x0                 (Alg 3 step 4, Eq. resi-local-domain-0)
//   threshold mask = |r0| > tau              (Sec. 2.3.1; or tau = beta max|r0|)
//   expansion unconditional graph layers, or Alg 3's conditional rounds
//   gradient  g_i = sum_j |x0_i - x0_j|      (Eq. grad; Alg 2)
//
// Every floating-point step that decides a set membership is the canonical
// serial order stated in include/lc_api.h, written with explicit
// round-to-nearest intrinsics so that the compiler can neither fuse nor
// reorder it; the masks are therefore bit-identical to a serial evaluation.
// Abs, max and the threshold tests run on the integer bit patterns.
#include <algorithm>
#include <cstdint>

#include "lc_internal.cuh"

namespace lc {

namespace {

constexpr int kResThreads = 256;   // 1024-cell chunk = 4 cells per thread

// Canonical residual of one stencil row: r = b_i, then r = fma(-a_ij, x_j, r)
// over j ascending (-z, -y, -x, P, +x, +y, +z); -a_ij = +T off the diagonal.
template <int DIM>
__device__ __forceinline__ double stencil_residual_row(const Stencil &op, const double *__restrict__ b,
                                                       const double *__restrict__ x, int64_t i) {
    const int64_t sxy = (int64_t)op.nx * op.ny;
    const unsigned ux = (unsigned)(i % op.nx);
    const unsigned uy = (unsigned)((i / op.nx) % op.ny);
    double r = b[i];
    if (DIM == 3) {
        const unsigned uz = (unsigned)(i / sxy);
        if (uz > 0) r = __fma_rn(op.Tz[i - sxy], x[i - sxy], r);
        if (uy > 0) r = __fma_rn(op.Ty[i - op.nx], x[i - op.nx], r);
        if (ux > 0) r = __fma_rn(op.Tx[i - 1], x[i - 1], r);
        r = __fma_rn(-op.D[i], x[i], r);
        if (ux + 1 < (unsigned)op.nx) r = __fma_rn(op.Tx[i], x[i + 1], r);
        if (uy + 1 < (unsigned)op.ny) r = __fma_rn(op.Ty[i], x[i + op.nx], r);
        if (uz + 1 < (unsigned)op.nz) r = __fma_rn(op.Tz[i], x[i + sxy], r);
    } else {
        if (uy > 0) r = __fma_rn(op.Ty[i - op.nx], x[i - op.nx], r);
        if (ux > 0) r = __fma_rn(op.Tx[i - 1], x[i - 1], r);
        r = __fma_rn(-op.D[i], x[i], r);
        if (ux + 1 < (unsigned)op.nx) r = __fma_rn(op.Tx[i], x[i + 1], r);
        if (uy + 1 < (unsigned)op.ny) r = __fma_rn(op.Ty[i], x[i + op.nx], r);
    }
    return r;
}

__device__ __forceinline__ double csr_residual_row(const Csr &op, const double *__restrict__ b,
                                                   const double *__restrict__ x, int32_t i) {
    double r = b[i];
    const int32_t e1 = op.rp[i + 1];
    for (int32_t e = op.rp[i]; e < e1; ++e) r = __fma_rn(-op.av[e], x[LC_IDX(op.ci[e], op.n)], r);
    return r;
}

// Sum of one 1024-value chunk held as v0..v3 = values t, t+256, t+512, t+768
// of the chunk, in the canonical stride-halving order (v[i] += v[i+s],
// s = 512 ... 1).  Returns the sum in thread 0.  blockDim.x must be 256.
__device__ __forceinline__ double chunk_tree(double v0, double v1, double v2, double v3, double *sm) {
    const int t = threadIdx.x;
    // s = 512: i = t (v0 += v2), i = t + 256 (v1 += v3)
    v0 = __dadd_rn(v0, v2);
    v1 = __dadd_rn(v1, v3);
    // s = 256: i = t < 256
    double v = __dadd_rn(v0, v1);
    sm[t] = v;
    __syncthreads();
    // s = 128, 64, 32 through shared memory
    for (int s = 128; s >= 32; s >>= 1) {
        if (t < s) sm[t] = __dadd_rn(sm[t], sm[t + s]);
        __syncthreads();
    }
    v = t < 32 ? sm[t] : 0.0;
    // s = 16 ... 1 inside warp 0
    if (t < 32) {
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            double w = __shfl_down_sync(kFull, v, s);
            v = __dadd_rn(v, w);
        }
    }
    __syncthreads();
    return v;
}

template <int DIM, bool TREE>
__global__ void __launch_bounds__(kResThreads) residual_stencil_kernel(Stencil op, const double *__restrict__ b,
                                                                       const double *__restrict__ x,
                                                                       double *__restrict__ r,
                                                                       double *__restrict__ partials, Ctrl *ctrl) {
    __shared__ double sm[kResThreads];
    __shared__ unsigned long long smx[32];
    const int64_t base = (int64_t)blockIdx.x * kTreeChunk;
    unsigned long long mx = 0;
    double sq[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = base + threadIdx.x + k * kResThreads;
        sq[k] = 0.0;
        if (i < op.n) {
            const double ri = stencil_residual_row<DIM>(op, b, x, i);
            r[i] = ri;
            const unsigned long long a = maxable_bits(ri);
            mx = a > mx ? a : mx;
            if (TREE) sq[k] = __dmul_rn(b[i], b[i]);
        }
    }
    mx = block_max(mx, smx);
    if (threadIdx.x == 0 && mx) atomicMax(&ctrl->maxabs_bits, mx);
    if (TREE) {
        const double s = chunk_tree(sq[0], sq[1], sq[2], sq[3], sm);
        if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
}

template <bool TREE>
__global__ void __launch_bounds__(kResThreads) residual_csr_kernel(Csr op, const double *__restrict__ b,
                                                                   const double *__restrict__ x,
                                                                   double *__restrict__ r,
                                                                   double *__restrict__ partials, Ctrl *ctrl) {
    __shared__ double sm[kResThreads];
    __shared__ unsigned long long smx[32];
    const int64_t base = (int64_t)blockIdx.x * kTreeChunk;
    unsigned long long mx = 0;
    double sq[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = base + threadIdx.x + k * kResThreads;
        sq[k] = 0.0;
        if (i < op.n) {
            const double ri = csr_residual_row(op, b, x, (int32_t)i);
            r[i] = ri;
            const unsigned long long a = maxable_bits(ri);
            mx = a > mx ? a : mx;
            if (TREE) sq[k] = __dmul_rn(b[i], b[i]);
        }
    }
    mx = block_max(mx, smx);
    if (threadIdx.x == 0 && mx) atomicMax(&ctrl->maxabs_bits, mx);
    if (TREE) {
        const double s = chunk_tree(sq[0], sq[1], sq[2], sq[3], sm);
        if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
}

// One further level of the canonical tree: chunk sums of `in` (m values).
__global__ void __launch_bounds__(kResThreads) tree_level_kernel(const double *__restrict__ in, int64_t m,
                                                                 double *__restrict__ out) {
    __shared__ double sm[kResThreads];
    const int64_t base = (int64_t)blockIdx.x * kTreeChunk;
    double v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = base + threadIdx.x + k * kResThreads;
        v[k] = i < m ? in[i] : 0.0;
    }
    const double s = chunk_tree(v[0], v[1], v[2], v[3], sm);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

__global__ void tau_eps_kernel(const double *S, int64_t n, double eps, Ctrl *ctrl, double *tau_out) {
    const double tau = __ddiv_rn(__dmul_rn(eps, __dsqrt_rn(*S)), __dsqrt_rn((double)n));
    ctrl->tau = tau;
    if (tau_out) *tau_out = tau;
}

__global__ void tau_relmax_kernel(double beta, Ctrl *ctrl, double *tau_out) {
    const double mx = __longlong_as_double((long long)ctrl->maxabs_bits);
    const double tau = __dmul_rn(beta, mx);
    ctrl->tau = tau;
    if (tau_out) *tau_out = tau;
}

__global__ void gmax_threshold_kernel(double alpha, Ctrl *ctrl, double *gmax_out) {
    const double gmax = __longlong_as_double((long long)ctrl->maxabs_bits);
    ctrl->tau = __dmul_rn(alpha, gmax);
    if (gmax_out) *gmax_out = gmax;
}

// Threshold and/or dilation on a structured grid through a shared-memory
// tile with a halo of `L` cells: flags of tile + halo are loaded (in-grid and
// |v| > tau, or the input mask), then L rounds of "add the face neighbours"
// run in shared memory on a region that shrinks by one cell per round.  The
// graph of a stencil operator with positive interior faces is the grid
// adjacency, so this is exactly L layers of graph dilation.
struct TileGeom {
    int tx, ty, tz;   // tile extent (cells)
    int L;            // halo = rounds in this pass
    int ex, ey, ez;   // extended extent
};

template <bool FROM_V>
__global__ void __launch_bounds__(256) threshold_dilate_kernel(Stencil op, TileGeom g, const double *__restrict__ v,
                                                               const uint8_t *__restrict__ mask_in,
                                                               uint8_t *__restrict__ mask_out, Ctrl *ctrl) {
    extern __shared__ uint8_t sflag[];
    uint8_t *f0 = sflag;
    uint8_t *f1 = sflag + g.ex * g.ey * g.ez;
    const int ntx = (op.nx + g.tx - 1) / g.tx, nty = (op.ny + g.ty - 1) / g.ty;
    const int bx = blockIdx.x % ntx;
    const int by = (blockIdx.x / ntx) % nty;
    const int bz = blockIdx.x / (ntx * nty);
    const int x0 = bx * g.tx - g.L, y0 = by * g.ty - g.L, z0 = bz * g.tz - (op.dim == 3 ? g.L : 0);
    const int ext = g.ex * g.ey * g.ez;
    unsigned long long tbits = 0;
    if (FROM_V) tbits = abs_bits(ctrl->tau);
    for (int k = threadIdx.x; k < ext; k += blockDim.x) {
        const int lx = k % g.ex, ly = (k / g.ex) % g.ey, lz = k / (g.ex * g.ey);
        const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
        uint8_t fl = 0;
        if (gx >= 0 && gx < op.nx && gy >= 0 && gy < op.ny && gz >= 0 && gz < op.nz) {
            const int64_t i = gx + (int64_t)op.nx * (gy + (int64_t)op.ny * gz);
            fl = FROM_V ? (uint8_t)abs_gt(v[i], tbits) : mask_in[i];
        }
        f0[k] = fl;
    }
    __syncthreads();
    for (int round = 1; round <= g.L; ++round) {
        for (int k = threadIdx.x; k < ext; k += blockDim.x) {
            const int lx = k % g.ex, ly = (k / g.ex) % g.ey, lz = k / (g.ex * g.ey);
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
            uint8_t o = f0[k];
            const bool inside = lx >= round && lx < g.ex - round && ly >= round && ly < g.ey - round &&
                                (op.dim == 2 || (lz >= round && lz < g.ez - round));
            if (inside && !o && gx >= 0 && gx < op.nx && gy >= 0 && gy < op.ny && gz >= 0 && gz < op.nz) {
                o = f0[k - 1] | f0[k + 1] | f0[k - g.ex] | f0[k + g.ex];
                if (op.dim == 3) o |= f0[k - g.ex * g.ey] | f0[k + g.ex * g.ey];
            }
            f1[k] = o;
        }
        __syncthreads();
        uint8_t *t = f0; f0 = f1; f1 = t;
    }
    const int tcells = g.tx * g.ty * g.tz;
    for (int k = threadIdx.x; k < tcells; k += blockDim.x) {
        const int lx = k % g.tx, ly = (k / g.tx) % g.ty, lz = k / (g.tx * g.ty);
        const int gx = x0 + g.L + lx, gy = y0 + g.L + ly, gz = z0 + (op.dim == 3 ? g.L : 0) + lz;
        if (gx < op.nx && gy < op.ny && gz < op.nz) {
            const int64_t i = gx + (int64_t)op.nx * (gy + (int64_t)op.ny * gz);
            const int e = (lx + g.L) + g.ex * ((ly + g.L) + g.ey * (lz + (op.dim == 3 ? g.L : 0)));
            mask_out[i] = f0[e];
        }
    }
}

// ---- bit-packed threshold and dilation (structured grids)
//
// The mask of a grid row (fixed y, z) as ceil(nx / 32) 32-bit words, bit b of
// word w = cell x = 32 w + b.  L rounds of the 4- (6-) neighbour dilation
// confined to the grid mark exactly the cells within L1 distance L of a
// marked cell -- a shortest lattice path between two cells of a box stays in
// the box -- so one pass ORs, for every row offset (dy, dz) with
// |dy| + |dz| <= L, the source row spread along x by L - |dy| - |dz| cells
// (funnel shifts across the neighbouring words).

// Threshold: bits of |v_i| > tau; a warp packs 32 words (1024 cells) of one row
// from coalesced loads, one ballot per word.
__global__ void __launch_bounds__(256) threshold_bits_kernel(Stencil op, int W, const double *__restrict__ v,
                                                             uint32_t *__restrict__ bits, Ctrl *ctrl) {
    const unsigned long long tbits = abs_bits(ctrl->tau);
    const int lane = threadIdx.x & 31;
    const int chunks = (W + 31) / 32;
    const int64_t tasks = (int64_t)op.ny * op.nz * chunks;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < tasks; t += nwarps) {
        const int64_t row = t / chunks;
        const int wx0 = (int)(t % chunks) * 32;
        const double *vr = v + row * op.nx;
        uint32_t mine = 0;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int x = (wx0 + k) * 32 + lane;
            const bool f = x < op.nx && abs_gt(vr[x], tbits);
            const uint32_t w = __ballot_sync(kFull, f);
            if (lane == k) mine = w;
        }
        if (wx0 + lane < W) bits[row * W + wx0 + lane] = mine;
    }
}

// One pass of L layers over the word rows: into words (BYTES false) or into
// the byte mask (BYTES true), one thread per word.
template <bool BYTES>
__global__ void __launch_bounds__(256) dilate_bits_kernel(Stencil op, int W, int L, const uint32_t *__restrict__ in,
                                                          uint32_t *__restrict__ out, uint8_t *__restrict__ mask,
                                                          int vec16) {
    const int64_t rows = (int64_t)op.ny * op.nz;
    const int64_t nw = rows * W;
    const int tail = op.nx & 31;
    const uint32_t last = tail ? (1u << tail) - 1u : 0xffffffffu;
    const int Lz = op.dim == 3 ? L : 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nw; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / W;
        const int wx = (int)(t - row * W);
        const int y = (int)(row % op.ny), z = (int)(row / op.ny);
        uint32_t o = 0;
        for (int dz = -Lz; dz <= Lz; ++dz) {
            const int zz = z + dz;
            if (zz < 0 || zz >= op.nz) continue;
            const int ry = L - (dz < 0 ? -dz : dz);
            for (int dy = -ry; dy <= ry; ++dy) {
                const int yy = y + dy;
                if (yy < 0 || yy >= op.ny) continue;
                const int r = ry - (dy < 0 ? -dy : dy);
                const uint32_t *src = in + ((int64_t)zz * op.ny + yy) * W + wx;
                const uint32_t c = src[0];
                uint32_t acc = c;
                if (r > 0) {
                    const uint32_t lft = wx > 0 ? src[-1] : 0u, rgt = wx + 1 < W ? src[1] : 0u;
                    for (int d = 1; d <= r; ++d)
                        acc |= __funnelshift_l(lft, c, d) | __funnelshift_r(c, rgt, d);
                }
                o |= acc;
            }
        }
        if (wx == W - 1) o &= last;
        if constexpr (!BYTES) {
            out[t] = o;
        } else {
            uint8_t *m = mask + row * op.nx + (int64_t)wx * 32;
            if (vec16 && wx < W - 1 + (tail == 0)) {   // 32 whole, 16-byte aligned cells
                uint32_t q[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) q[k] = (((o >> (4 * k)) & 15u) * 0x00204081u) & 0x01010101u;
                reinterpret_cast<uint4 *>(m)[0] = make_uint4(q[0], q[1], q[2], q[3]);
                reinterpret_cast<uint4 *>(m)[1] = make_uint4(q[4], q[5], q[6], q[7]);
            } else {
                const int nb = min(32, op.nx - wx * 32);
                for (int k = 0; k < nb; ++k) m[k] = (uint8_t)((o >> k) & 1u);
            }
        }
    }
}

__global__ void threshold_flat_kernel(int64_t n, const double *__restrict__ v, uint8_t *__restrict__ mask, Ctrl *ctrl) {
    const unsigned long long tbits = abs_bits(ctrl->tau);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mask[i] = (uint8_t)abs_gt(v[i], tbits);
}

__global__ void dilate_csr_kernel(Csr op, const uint8_t *__restrict__ in, uint8_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < op.n; i += (int64_t)gridDim.x * blockDim.x) {
        uint8_t m = in[i];
        if (!m) {
            const int32_t e1 = op.rp[i + 1];
            for (int32_t e = op.rp[i]; e < e1; ++e) {
                const int32_t j = LC_IDX(op.ci[e], op.n);
                if (j != i && op.av[e] != 0.0 && in[j]) { m = 1; break; }
            }
        }
        out[i] = m;
    }
}

// One synchronous round of Alg 3: a point j outside the domain whose row
// couples it to the domain is added when |r0_j| + t > tau, with
// t = sum over domain neighbours i (ascending) of |fl(a_ji * x0_i)|.
template <int DIM>
__global__ void __launch_bounds__(256) expand_paper_stencil_kernel(Stencil op, const double *__restrict__ r,
                                                                   const double *__restrict__ x0, int round,
                                                                   const uint8_t *__restrict__ in,
                                                                   uint8_t *__restrict__ out, Ctrl *ctrl) {
    __shared__ int sm[32];
    const bool skip = round > 0 && *(volatile int32_t *)&ctrl->added[round - 1] == 0;
    const unsigned long long tbits = abs_bits(ctrl->tau);
    const int64_t sxy = (int64_t)op.nx * op.ny;
    int added = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < op.n; j += (int64_t)gridDim.x * blockDim.x) {
        uint8_t m = in[j];
        if (!m && !skip) {
            // coordinates in 32-bit arithmetic (N < 2^31), the face and x0 of a
            // neighbour read only when it is in the domain
            const unsigned uj = (unsigned)j, unx = (unsigned)op.nx;
            const unsigned ux = uj % unx;
            const unsigned uy = (uj / unx) % (unsigned)op.ny;
            const unsigned uz = DIM == 3 ? uj / (unsigned)sxy : 0u;
            bool nbr = false;
            double t = 0.0;
            auto visit = [&](bool ok, int64_t i, const double *T, int64_t f) {
                if (ok && in[i]) {
                    nbr = true;
                    t = __dadd_rn(t, fabs(__dmul_rn(T[f], x0[i])));
                }
            };
            if (DIM == 3) visit(uz > 0, j - sxy, op.Tz, j - sxy);
            visit(uy > 0, j - op.nx, op.Ty, j - op.nx);
            visit(ux > 0, j - 1, op.Tx, j - 1);
            visit(ux + 1 < unx, j + 1, op.Tx, j);
            visit(uy + 1 < (unsigned)op.ny, j + op.nx, op.Ty, j);
            if (DIM == 3) visit(uz + 1 < (unsigned)op.nz, j + sxy, op.Tz, j);
            if (nbr) {
                const double c = __dadd_rn(fabs(r[j]), t);
                if (abs_gt(c, tbits)) { m = 1; ++added; }
            }
        }
        out[j] = m;
    }
    added = block_isum(added, sm);
    if (threadIdx.x == 0 && added) atomicAdd(&ctrl->added[round], added);
}

__global__ void __launch_bounds__(256) expand_paper_csr_kernel(Csr op, const double *__restrict__ r,
                                                               const double *__restrict__ x0, int round,
                                                               const uint8_t *__restrict__ in,
                                                               uint8_t *__restrict__ out, Ctrl *ctrl) {
    __shared__ int sm[32];
    const bool skip = round > 0 && *(volatile int32_t *)&ctrl->added[round - 1] == 0;
    const unsigned long long tbits = abs_bits(ctrl->tau);
    int added = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < op.n; j += (int64_t)gridDim.x * blockDim.x) {
        uint8_t m = in[j];
        if (!m && !skip) {
            bool nbr = false;
            double t = 0.0;
            const int32_t e1 = op.rp[j + 1];
            for (int32_t e = op.rp[j]; e < e1; ++e) {
                const int32_t i = LC_IDX(op.ci[e], op.n);
                if (i == j || !in[i]) continue;
                if (op.av[e] != 0.0) nbr = true;
                t = __dadd_rn(t, fabs(__dmul_rn(op.av[e], x0[i])));
            }
            if (nbr) {
                const double c = __dadd_rn(fabs(r[j]), t);
                if (abs_gt(c, tbits)) { m = 1; ++added; }
            }
        }
        out[j] = m;
    }
    added = block_isum(added, sm);
    if (threadIdx.x == 0 && added) atomicAdd(&ctrl->added[round], added);
}

// g_i = 0; g_i = g_i + |x_i - x_j| over neighbours j ascending.
template <int DIM>
__global__ void __launch_bounds__(256) gradient_stencil_kernel(Stencil op, const double *__restrict__ x,
                                                               double *__restrict__ g, Ctrl *ctrl) {
    __shared__ unsigned long long smx[32];
    const int64_t sxy = (int64_t)op.nx * op.ny;
    unsigned long long mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < op.n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned ux = (unsigned)(i % op.nx);
        const unsigned uy = (unsigned)((i / op.nx) % op.ny);
        const unsigned uz = DIM == 3 ? (unsigned)(i / sxy) : 0u;
        const double xi = x[i];
        double s = 0.0;
        if (DIM == 3 && uz > 0) s = __dadd_rn(s, fabs(__dsub_rn(xi, x[i - sxy])));
        if (uy > 0) s = __dadd_rn(s, fabs(__dsub_rn(xi, x[i - op.nx])));
        if (ux > 0) s = __dadd_rn(s, fabs(__dsub_rn(xi, x[i - 1])));
        if (ux + 1 < (unsigned)op.nx) s = __dadd_rn(s, fabs(__dsub_rn(xi, x[i + 1])));
        if (uy + 1 < (unsigned)op.ny) s = __dadd_rn(s, fabs(__dsub_rn(xi, x[i + op.nx])));
        if (DIM == 3 && uz + 1 < (unsigned)op.nz) s = __dadd_rn(s, fabs(__dsub_rn(xi, x[i + sxy])));
        g[i] = s;
        const unsigned long long a = maxable_bits(s);
        mx = a > mx ? a : mx;
    }
    mx = block_max(mx, smx);
    if (threadIdx.x == 0 && mx) atomicMax(&ctrl->maxabs_bits, mx);
}

__global__ void __launch_bounds__(256) gradient_csr_kernel(Csr op, const double *__restrict__ x, double *__restrict__ g,
                                                           Ctrl *ctrl) {
    __shared__ unsigned long long smx[32];
    unsigned long long mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < op.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double xi = x[i];
        double s = 0.0;
        const int32_t e1 = op.rp[i + 1];
        for (int32_t e = op.rp[i]; e < e1; ++e) {
            const int32_t j = LC_IDX(op.ci[e], op.n);
            if (j == i || op.av[e] == 0.0) continue;
            s = __dadd_rn(s, fabs(__dsub_rn(xi, x[j])));
        }
        g[i] = s;
        const unsigned long long a = maxable_bits(s);
        mx = a > mx ? a : mx;
    }
    mx = block_max(mx, smx);
    if (threadIdx.x == 0 && mx) atomicMax(&ctrl->maxabs_bits, mx);
}

__global__ void __launch_bounds__(256) count_mask_kernel(int64_t n, const uint8_t *__restrict__ mask, Ctrl *ctrl) {
    __shared__ int sm[32];
    int c = 0;
    const int64_t n16 = ((uintptr_t)mask & 15) ? 0 : n / 16;   // vector path needs 16-byte alignment
    const uint4 *m16 = reinterpret_cast<const uint4 *>(mask);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n16; k += (int64_t)gridDim.x * blockDim.x) {
        const uint4 w = m16[k];
        c += __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);   // mask bytes are 0 or 1
    }
    for (int64_t i = n16 * 16 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        c += mask[i];
    c = block_isum(c, sm);
    if (threadIdx.x == 0 && c) atomicAdd(&ctrl->K, c);
}

__global__ void copy_k_kernel(const Ctrl *ctrl, int32_t *K_out) { *K_out = ctrl->K; }

inline int flat_grid(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_residual_stencil(const Stencil &op, const double *b, const double *x, double *r, int want_tree,
                                    double *tree_partials, Ctrl *ctrl, cudaStream_t s) {
    const int nb = (int)((op.n + kTreeChunk - 1) / kTreeChunk);
    if (op.dim == 3) {
        if (want_tree) { residual_stencil_kernel<3, true><<<nb, kResThreads, 0, s>>>(op, b, x, r, tree_partials, ctrl); note_launches(1); }
        else { residual_stencil_kernel<3, false><<<nb, kResThreads, 0, s>>>(op, b, x, r, tree_partials, ctrl); note_launches(1); }
    } else {
        if (want_tree) { residual_stencil_kernel<2, true><<<nb, kResThreads, 0, s>>>(op, b, x, r, tree_partials, ctrl); note_launches(1); }
        else { residual_stencil_kernel<2, false><<<nb, kResThreads, 0, s>>>(op, b, x, r, tree_partials, ctrl); note_launches(1); }
    }
    return cudaGetLastError();
}

cudaError_t launch_residual_csr(const Csr &op, const double *b, const double *x, double *r, int want_tree,
                                double *tree_partials, Ctrl *ctrl, cudaStream_t s) {
    const int nb = (int)((op.n + kTreeChunk - 1) / kTreeChunk);
    if (want_tree) { residual_csr_kernel<true><<<nb, kResThreads, 0, s>>>(op, b, x, r, tree_partials, ctrl); note_launches(1); }
    else { residual_csr_kernel<false><<<nb, kResThreads, 0, s>>>(op, b, x, r, tree_partials, ctrl); note_launches(1); }
    return cudaGetLastError();
}

// Reduce the chunk sums level by level (ping-pong between partials and
// scratch, each at least ceil(n/1024) long) and form tau.
cudaError_t launch_tree_finish(double *partials, double *scratch, int64_t nchunks, int64_t n, double eps, Ctrl *ctrl,
                               double *tau_out, cudaStream_t s) {
    double *in = partials, *out = scratch;
    int64_t m = nchunks;
    while (m > 1) {
        const int64_t nb = (m + kTreeChunk - 1) / kTreeChunk;
        tree_level_kernel<<<(unsigned)nb, kResThreads, 0, s>>>(in, m, out);
        note_launches(1);
        double *t = in; in = out; out = t;
        m = nb;
    }
    tau_eps_kernel<<<1, 1, 0, s>>>(in, n, eps, ctrl, tau_out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tau_relmax(double beta, Ctrl *ctrl, double *tau_out, cudaStream_t s) {
    tau_relmax_kernel<<<1, 1, 0, s>>>(beta, ctrl, tau_out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gmax_threshold(double alpha, Ctrl *ctrl, double *gmax_out, cudaStream_t s) {
    gmax_threshold_kernel<<<1, 1, 0, s>>>(alpha, ctrl, gmax_out);
    note_launches(1);
    return cudaGetLastError();
}

// One pass: threshold v against ctrl->tau, then `layers` (<= max_layers_per_pass)
// graph layers, writing `mask`.  Further layers use launch_dilate_stencil_pass.
cudaError_t launch_threshold_dilate_stencil(const Stencil &op, const double *v, int layers, uint8_t *mask, Ctrl *ctrl,
                                            cudaStream_t s) {
    TileGeom g;
    if (op.dim == 3) { g.tx = 16; g.ty = 8; g.tz = 8; }
    else { g.tx = 64; g.ty = 16; g.tz = 1; }
    g.L = layers;
    g.ex = g.tx + 2 * layers;
    g.ey = g.ty + 2 * layers;
    g.ez = op.dim == 3 ? g.tz + 2 * layers : 1;
    const int ntx = (op.nx + g.tx - 1) / g.tx, nty = (op.ny + g.ty - 1) / g.ty, ntz = (op.nz + g.tz - 1) / g.tz;
    const size_t smem = 2 * (size_t)g.ex * g.ey * g.ez;
    const unsigned nb = (unsigned)((int64_t)ntx * nty * ntz);
    threshold_dilate_kernel<true><<<nb, 256, smem, s>>>(op, g, v, nullptr, mask, ctrl);
    note_launches(1);
    return cudaGetLastError();
}

int bits_words(const Stencil &op) { return (op.nx + 31) / 32; }

cudaError_t launch_threshold_dilate_bits(const Stencil &op, const double *v, int layers, uint8_t *mask,
                                         uint32_t *bits_a, uint32_t *bits_b, Ctrl *ctrl, cudaStream_t s) {
    const int W = bits_words(op);
    const int64_t rows = (int64_t)op.ny * op.nz;
    const int64_t tasks = rows * ((W + 31) / 32);
    const unsigned nba = (unsigned)std::min<int64_t>((tasks + 7) / 8, 152 * 16);
    threshold_bits_kernel<<<nba, 256, 0, s>>>(op, W, v, bits_a, ctrl);
    note_launches(1);
    const int lmax = op.dim == 3 ? 4 : 8;   // layers per pass: the pass costs O(L^dim) word operations
    const unsigned nbb = (unsigned)std::min<int64_t>((rows * W + 255) / 256, 152 * 16);
    const int vec16 = (op.nx % 16 == 0) && ((reinterpret_cast<uintptr_t>(mask) & 15) == 0);
    const uint32_t *cur = bits_a;
    uint32_t *nxt = bits_b;
    int left = layers;
    while (left > lmax) {
        dilate_bits_kernel<false><<<nbb, 256, 0, s>>>(op, W, lmax, cur, nxt, nullptr, 0);
        note_launches(1);
        left -= lmax;
        uint32_t *t = const_cast<uint32_t *>(cur);
        cur = nxt;
        nxt = t;
    }
    dilate_bits_kernel<true><<<nbb, 256, 0, s>>>(op, W, left, cur, nullptr, mask, vec16);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dilate_stencil_pass(const Stencil &op, int layers, const uint8_t *in, uint8_t *out, cudaStream_t s) {
    TileGeom g;
    if (op.dim == 3) { g.tx = 16; g.ty = 8; g.tz = 8; }
    else { g.tx = 64; g.ty = 16; g.tz = 1; }
    g.L = layers;
    g.ex = g.tx + 2 * layers;
    g.ey = g.ty + 2 * layers;
    g.ez = op.dim == 3 ? g.tz + 2 * layers : 1;
    const int ntx = (op.nx + g.tx - 1) / g.tx, nty = (op.ny + g.ty - 1) / g.ty, ntz = (op.nz + g.tz - 1) / g.tz;
    const size_t smem = 2 * (size_t)g.ex * g.ey * g.ez;
    const unsigned nb = (unsigned)((int64_t)ntx * nty * ntz);
    threshold_dilate_kernel<false><<<nb, 256, smem, s>>>(op, g, nullptr, in, out, nullptr);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_threshold_csr(int32_t n, const double *v, uint8_t *mask, Ctrl *ctrl, cudaStream_t s) {
    threshold_flat_kernel<<<flat_grid(n), 256, 0, s>>>(n, v, mask, ctrl);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dilate_csr(const Csr &op, const uint8_t *in, uint8_t *out, cudaStream_t s) {
    dilate_csr_kernel<<<flat_grid(op.n), 256, 0, s>>>(op, in, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_expand_paper_stencil(const Stencil &op, const double *r, const double *x0, int round,
                                        const uint8_t *in, uint8_t *out, Ctrl *ctrl, cudaStream_t s) {
    if (op.dim == 3) { expand_paper_stencil_kernel<3><<<flat_grid(op.n), 256, 0, s>>>(op, r, x0, round, in, out, ctrl); note_launches(1); }
    else { expand_paper_stencil_kernel<2><<<flat_grid(op.n), 256, 0, s>>>(op, r, x0, round, in, out, ctrl); note_launches(1); }
    return cudaGetLastError();
}

cudaError_t launch_expand_paper_csr(const Csr &op, const double *r, const double *x0, int round, const uint8_t *in,
                                    uint8_t *out, Ctrl *ctrl, cudaStream_t s) {
    expand_paper_csr_kernel<<<flat_grid(op.n), 256, 0, s>>>(op, r, x0, round, in, out, ctrl);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gradient_stencil(const Stencil &op, const double *x, double *g, Ctrl *ctrl, cudaStream_t s) {
    if (op.dim == 3) { gradient_stencil_kernel<3><<<flat_grid(op.n), 256, 0, s>>>(op, x, g, ctrl); note_launches(1); }
    else { gradient_stencil_kernel<2><<<flat_grid(op.n), 256, 0, s>>>(op, x, g, ctrl); note_launches(1); }
    return cudaGetLastError();
}

cudaError_t launch_gradient_csr(const Csr &op, const double *x, double *g, Ctrl *ctrl, cudaStream_t s) {
    gradient_csr_kernel<<<flat_grid(op.n), 256, 0, s>>>(op, x, g, ctrl);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_count_mask(int64_t n, const uint8_t *mask, Ctrl *ctrl, int32_t *K_out, cudaStream_t s) {
    count_mask_kernel<<<flat_grid((n + 15) / 16), 256, 0, s>>>(n, mask, ctrl);
    note_launches(1);
    if (K_out) { copy_k_kernel<<<1, 1, 0, s>>>(ctrl, K_out); note_launches(1); }
    return cudaGetLastError();
}

}  // namespace lc
