// lc_batched.cu -- many independent 2D systems, each solved by Alg 1 end to
// end, in ONE persistent launch (captured in a CUDA graph by lc_api.cu).
//
// Every CTA takes systems from a device work queue (largest first) and runs,
// with block-level synchronisation only (systems are independent, so there
// is no grid-wide wait):
//   residual marking  r0 = b - A x0 in the canonical order, tau = beta max|r0|,
//                     mask = |r0| > tau, `layers` rounds of dilation  (Alg 3 variant)
//   extraction        packed-pair block scan -> g2l, l2g, rowptr; B, rhs, xL0  (Eq. loc-equ)
//   local solve       iterative refinement: FP64 residual, FP32 Jacobi-CG on fl32(B)
//   assembly          x~ = x0 with x~[l2g] = xL                               (Eq. sol-assemble)
//   check + global    iterative refinement on the whole system from x~; returns at once
//                     if ||b - A x~|| <= tol ||b||                            (Alg 1 steps 8-11)
// The masks and subsystems are bit-identical to lc_mark_residual / lc_extract
// on the same system (same canonical orders); the solves reach the same FP64
// relative residual.
#include "lc_internal.cuh"

namespace lc {

namespace {

template <int BS>
struct Blk {
    double *red;   // shared scratch, >= 4 * 32 doubles
    __device__ double sum(double v) const {
        double a[1] = {v};
        block_sum<1, double>(a, red);
        if (threadIdx.x == 0) red[96] = a[0];
        __syncthreads();
        const double r = red[96];
        __syncthreads();
        return r;
    }
    __device__ void sum2(double &u, double &v) const {
        double a[2] = {u, v};
        block_sum<2, double>(a, red);
        if (threadIdx.x == 0) { red[96] = a[0]; red[97] = a[1]; }
        __syncthreads();
        u = red[96];
        v = red[97];
        __syncthreads();
    }
    __device__ void sum2f(float &u, float &v) const {
        float a[2] = {u, v};
        block_sum<2, float>(a, reinterpret_cast<float *>(red));
        if (threadIdx.x == 0) { red[96] = a[0]; red[97] = a[1]; }
        __syncthreads();
        u = (float)red[96];
        v = (float)red[97];
        __syncthreads();
    }
};

// exclusive scan of one packed pair per thread over the block; returns the
// prefix and the block total (all threads)
__device__ __forceinline__ unsigned long long blk_scan(unsigned long long v, unsigned long long *sm,
                                                       unsigned long long &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long w = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += w;
    }
    __syncthreads();
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? sm[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) sm[lane] = w;
    }
    __syncthreads();
    total = sm[nw - 1];
    return (warp > 0 ? sm[warp - 1] : 0ull) + inc - v;
}

// one system -----------------------------------------------------------------

struct Sys {
    int nx, ny, n;
    int64_t o;     // cell offset
    int64_t oe;    // offset of B's entries (5 o)
    int64_t orp;   // offset of B's row pointers (o + s)
};

// canonical residual of cell i (local index), FP64
__device__ __forceinline__ double res_row(const BatchView &V, const Sys &S, const double *x, int i) {
    const int ux = i % S.nx, uy = i / S.nx;
    const int64_t g = S.o + i;
    double r = V.b[g];
    if (uy > 0) r = __fma_rn(V.Ty[g - S.nx], x[g - S.nx], r);
    if (ux > 0) r = __fma_rn(V.Tx[g - 1], x[g - 1], r);
    r = __fma_rn(-V.D[g], x[g], r);
    if (ux + 1 < S.nx) r = __fma_rn(V.Tx[g], x[g + 1], r);
    if (uy + 1 < S.ny) r = __fma_rn(V.Ty[g], x[g + S.nx], r);
    return r;
}

// q = A32 p on the FP32 stencil (local index i)
__device__ __forceinline__ float spmv32(const BatchView &V, const Sys &S, const float *p, int i) {
    const int ux = i % S.nx, uy = i / S.nx;
    const int64_t g = S.o + i;
    float q = V.D32[g] * p[g];
    if (uy > 0) q = fmaf(-V.Ty32[g - S.nx], p[g - S.nx], q);
    if (ux > 0) q = fmaf(-V.Tx32[g - 1], p[g - 1], q);
    if (ux + 1 < S.nx) q = fmaf(-V.Tx32[g], p[g + 1], q);
    if (uy + 1 < S.ny) q = fmaf(-V.Ty32[g], p[g + S.nx], q);
    return q;
}

// Reduction asked of a sweep's inner solve: inner_tol, or -- when the outer
// test (rr <= stop) misses by less -- half of what is still missing.
__device__ __forceinline__ double sweep_tol(double inner_tol, double stop, double rr) {
    const double need = 0.5 * sqrt(stop / rr);
    return need > inner_tol ? need : inner_tol;
}

// FP32 Jacobi-CG on (A32 | B32) d = r32 from d = 0 over `n` unknowns at `o`
// (cells of the system, or rows of its subsystem); stops when the residual
// fell by inner_tol or after max_inner iterations.  Returns iterations.
// Each thread takes its unknowns two at a time (i, i + BS) and issues both
// unknowns' loads before either one's stores: a store whose value waits on
// a load would otherwise hold every later load back (the compiler cannot
// prove the arrays apart), one memory latency per unknown.  Sums keep the
// order i, i + BS, i + 2 BS, ... of a plain strided loop.  (Measured on the
// 512-system batch: one unknown per trip 28.3 ms, two 21.6 ms; generic
// loops over 2, 4 or 8 unknowns came out between 21.3 and 27.5 ms, and
// slower on the small multi-group systems.)
template <int BS, bool CSR>
__device__ int inner_cg(const BatchView &V, const Sys &S, const Blk<BS> &blk, int n, int64_t o, const float *dinv,
                        double inner_tol, int max_inner, int &breakdown) {
    float *r = V.r32 + o, *z = V.z32 + o, *p = V.p32 + o, *q = V.q32 + o, *d = V.d32 + o;
    auto aq = [&](int i) {   // (A p)_i or (B p)_i
        if (CSR) {
            float qi = 0.f;
            const int32_t e0 = V.rowptr[S.orp + i], e1 = V.rowptr[S.orp + i + 1];
            for (int32_t e = e0; e < e1; ++e) qi = fmaf(V.val32[S.oe + e], p[V.col[S.oe + e]], qi);
            return qi;
        } else {
            return spmv32(V, S, V.p32, i);
        }
    };
    float rz = 0.f, rr = 0.f;
    for (int i = threadIdx.x; i < n; i += 2 * BS) {
        const int j = i + BS;
        const bool two = j < n;
        const float ri = r[i], di = dinv[i];
        float rj = 0.f, dj = 0.f;
        if (two) { rj = r[j]; dj = dinv[j]; }
        const float zi = di * ri, zj = dj * rj;
        d[i] = 0.f; z[i] = zi; p[i] = zi;
        rz = fmaf(ri, zi, rz);
        rr = fmaf(ri, ri, rr);
        if (two) {
            d[j] = 0.f; z[j] = zj; p[j] = zj;
            rz = fmaf(rj, zj, rz);
            rr = fmaf(rj, rj, rr);
        }
    }
    blk.sum2f(rz, rr);
    const float stop = (float)(inner_tol * inner_tol) * rr;
    int it = 0;
    while (it < max_inner && rr > stop) {
        float pq = 0.f;
        for (int i = threadIdx.x; i < n; i += 2 * BS) {
            const int j = i + BS;
            const bool two = j < n;
            const float qi = aq(i), pi = p[i];
            float qj = 0.f, pj = 0.f;
            if (two) { qj = aq(j); pj = p[j]; }
            q[i] = qi;
            pq = fmaf(pi, qi, pq);
            if (two) { q[j] = qj; pq = fmaf(pj, qj, pq); }
        }
        float dummy = 0.f;
        blk.sum2f(pq, dummy);
        if (!(pq > 0.f) || !isfinite(pq)) { breakdown = 1; break; }
        const float alpha = rz / pq;
        float rz2 = 0.f, rr2 = 0.f;
        for (int i = threadIdx.x; i < n; i += 2 * BS) {
            const int j = i + BS;
            const bool two = j < n;
            const float pi = p[i], di = d[i], qi = q[i], r0i = r[i], vi = dinv[i];
            float pj = 0.f, dj = 0.f, qj = 0.f, r0j = 0.f, vj = 0.f;
            if (two) { pj = p[j]; dj = d[j]; qj = q[j]; r0j = r[j]; vj = dinv[j]; }
            const float ri = fmaf(-alpha, qi, r0i), zi = vi * ri;
            d[i] = fmaf(alpha, pi, di);
            r[i] = ri;
            z[i] = zi;
            rz2 = fmaf(ri, zi, rz2);
            rr2 = fmaf(ri, ri, rr2);
            if (two) {
                const float rj = fmaf(-alpha, qj, r0j), zj = vj * rj;
                d[j] = fmaf(alpha, pj, dj);
                r[j] = rj;
                z[j] = zj;
                rz2 = fmaf(rj, zj, rz2);
                rr2 = fmaf(rj, rj, rr2);
            }
        }
        blk.sum2f(rz2, rr2);
        ++it;
        const float beta = rz2 / rz;
        rz = rz2;
        rr = rr2;
        for (int i = threadIdx.x; i < n; i += 2 * BS) {
            const int j = i + BS;
            const bool two = j < n;
            const float pi = p[i], zi = z[i];
            float pj = 0.f, zj = 0.f;
            if (two) { pj = p[j]; zj = z[j]; }
            p[i] = fmaf(beta, pi, zi);
            if (two) p[j] = fmaf(beta, pj, zj);
        }
        __syncthreads();
    }
    return it;
}

template <int BS>
__device__ void solve_system(const BatchView &V, const BatchParams &P, int s, const Blk<BS> &blk,
                             unsigned long long *scan_sm) {
    Sys S;
    S.nx = V.nx[s];
    S.ny = V.ny[s];
    S.n = S.nx * S.ny;
    S.o = V.off[s];
    S.oe = 5 * S.o;
    S.orp = S.o + s;
    const int n = S.n;
    int32_t *st = V.stat_i + 8 * (int64_t)s;
    double *sd = V.stat_d + 4 * (int64_t)s;
    int breakdown = 0;

    // ---- residual marking (canonical residual, relative threshold, layers)
    unsigned long long mx = 0;
    for (int i = threadIdx.x; i < n; i += 2 * BS) {   // two cells at a time, loads before stores
        const int j = i + BS;
        const double ri = res_row(V, S, V.x, i);
        const double rj = j < n ? res_row(V, S, V.x, j) : 0.0;
        V.r[S.o + i] = ri;
        unsigned long long a = maxable_bits(ri);
        mx = a > mx ? a : mx;
        if (j < n) {
            V.r[S.o + j] = rj;
            a = maxable_bits(rj);
            mx = a > mx ? a : mx;
        }
    }
    mx = block_max(mx, scan_sm);
    if (threadIdx.x == 0) scan_sm[40] = mx;
    __syncthreads();
    const double tau = __dmul_rn(P.beta, __longlong_as_double((long long)scan_sm[40]));
    __syncthreads();
    const unsigned long long tbits = abs_bits(tau);
    uint8_t *ma = V.m0 + S.o, *mb = V.m1 + S.o;
    for (int i = threadIdx.x; i < n; i += BS) ma[i] = (uint8_t)abs_gt(V.r[S.o + i], tbits);
    __syncthreads();
    for (int l = 0; l < P.layers; ++l) {
        for (int i = threadIdx.x; i < n; i += BS) {
            const int ux = i % S.nx, uy = i / S.nx;
            uint8_t m = ma[i];
            if (!m) m = (uy > 0 && ma[i - S.nx]) | (ux > 0 && ma[i - 1]) | (ux + 1 < S.nx && ma[i + 1]) |
                        (uy + 1 < S.ny && ma[i + S.nx]);
            mb[i] = m;
        }
        __syncthreads();
        uint8_t *t = ma; ma = mb; mb = t;
    }

    // ---- compaction: one packed (cells, entries) scan over the cells in order
    int32_t *g2l = V.g2l + S.o, *l2g = V.l2g + S.o, *rp = V.rowptr + S.orp;
    unsigned long long run = 0;
    for (int base = 0; base < n; base += BS) {
        const int i = base + threadIdx.x;
        unsigned long long v = 0;
        if (i < n && ma[i]) {
            const int ux = i % S.nx, uy = i / S.nx;
            unsigned c = 1;
            if (uy > 0) c += ma[i - S.nx];
            if (ux > 0) c += ma[i - 1];
            if (ux + 1 < S.nx) c += ma[i + 1];
            if (uy + 1 < S.ny) c += ma[i + S.nx];
            v = 1ull | ((unsigned long long)c << 32);
        }
        unsigned long long tot;
        const unsigned long long pre = blk_scan(v, scan_sm, tot) + run;
        if (i < n) {
            if (v) {
                const int32_t l = (int32_t)(pre & 0xffffffffull);
                g2l[i] = l;
                l2g[l] = i;
                rp[l] = (int32_t)(pre >> 32);
            } else {
                g2l[i] = -1;
            }
        }
        run += tot;
    }
    const int K = (int)(run & 0xffffffffull);
    const int nzB = (int)(run >> 32);
    if (threadIdx.x == 0) rp[K] = nzB;
    __syncthreads();

    // ---- gather B (FP64 and FP32 values), rhs (canonical order), xL0, 1/diag
    for (int l = threadIdx.x; l < K; l += BS) {
        const int i = l2g[l];
        const int ux = i % S.nx, uy = i / S.nx;
        const int64_t g = S.o + i;
        int32_t e = rp[l];
        double sacc = V.b[g];
        auto visit = [&](int j, double T) {
            const int32_t gj = g2l[j];
            if (gj >= 0) { V.col[S.oe + e] = gj; V.val[S.oe + e] = -T; V.val32[S.oe + e] = (float)-T; ++e; }
            else sacc = __fma_rn(T, V.x[S.o + j], sacc);
        };
        if (uy > 0) visit(i - S.nx, V.Ty[g - S.nx]);
        if (ux > 0) visit(i - 1, V.Tx[g - 1]);
        V.col[S.oe + e] = l; V.val[S.oe + e] = V.D[g]; V.val32[S.oe + e] = (float)V.D[g]; ++e;
        if (ux + 1 < S.nx) visit(i + 1, V.Tx[g]);
        if (uy + 1 < S.ny) visit(i + S.nx, V.Ty[g]);
        V.rhs[S.o + l] = sacc;
        V.xl[S.o + l] = V.x[g];
        V.dl32[S.o + l] = 1.0f / (float)V.D[g];
    }
    __syncthreads();

    // ---- local solve: iterative refinement on B (FP64 residual, FP32 CG)
    int it_l = 0, outer_l = 0;
    if (K > 0) {
        double bb = 0.0;
        for (int l = threadIdx.x; l < K; l += BS) bb = fma(V.rhs[S.o + l], V.rhs[S.o + l], bb);
        bb = blk.sum(bb);
        const double stop = (P.tol_local * P.tol_local) * bb;
        while (true) {
            double rr = 0.0;
            for (int l = threadIdx.x; l < K; l += BS) {
                double a = 0.0;
                const int32_t e1 = rp[l + 1];
                for (int32_t e = rp[l]; e < e1; ++e) a = fma(V.val[S.oe + e], V.xl[S.o + V.col[S.oe + e]], a);
                const double rl = V.rhs[S.o + l] - a;
                V.r[S.o + l] = rl;
                rr = fma(rl, rl, rr);
            }
            rr = blk.sum(rr);
            if (rr <= stop || bb == 0.0 || outer_l >= P.max_outer) break;
            const double sc = sqrt(rr), inv = 1.0 / sc;
            for (int l = threadIdx.x; l < K; l += BS) V.r32[S.o + l] = (float)(V.r[S.o + l] * inv);
            __syncthreads();
            it_l += inner_cg<BS, true>(V, S, blk, K, S.o, V.dl32 + S.o, sweep_tol(P.inner_tol, stop, rr), P.max_inner,
                                       breakdown);
            for (int l = threadIdx.x; l < K; l += BS) V.xl[S.o + l] = fma(sc, (double)V.d32[S.o + l], V.xl[S.o + l]);
            __syncthreads();
            ++outer_l;
            if (breakdown) break;
        }
    }
    // ---- assembly x~ = x0 with the local solution
    for (int l = threadIdx.x; l < K; l += BS) V.x[S.o + l2g[l]] = V.xl[S.o + l];
    __syncthreads();

    // ---- check of x~ and global solve: iterative refinement on A
    int it_g = 0, outer_g = 0;
    double bb = 0.0, rr0 = 0.0, rr = 0.0;
    for (int i = threadIdx.x; i < n; i += BS) bb = fma(V.b[S.o + i], V.b[S.o + i], bb);
    bb = blk.sum(bb);
    const double stop = (P.tol * P.tol) * bb;
    while (true) {
        rr = 0.0;
        for (int i = threadIdx.x; i < n; i += 2 * BS) {   // two cells at a time, loads before stores
            const int j = i + BS;
            const double ri = res_row(V, S, V.x, i);
            const double rj = j < n ? res_row(V, S, V.x, j) : 0.0;
            V.r[S.o + i] = ri;
            rr = fma(ri, ri, rr);
            if (j < n) {
                V.r[S.o + j] = rj;
                rr = fma(rj, rj, rr);
            }
        }
        rr = blk.sum(rr);
        if (outer_g == 0) rr0 = rr;
        if (rr <= stop || bb == 0.0 || outer_g >= P.max_outer || breakdown) break;
        const double sc = sqrt(rr), inv = 1.0 / sc;
        for (int i = threadIdx.x; i < n; i += 2 * BS) {
            const int j = i + BS;
            const double ri = V.r[S.o + i], rj = j < n ? V.r[S.o + j] : 0.0;
            V.r32[S.o + i] = (float)(ri * inv);
            if (j < n) V.r32[S.o + j] = (float)(rj * inv);
        }
        __syncthreads();
        it_g += inner_cg<BS, false>(V, S, blk, n, S.o, V.dinv32 + S.o, sweep_tol(P.inner_tol, stop, rr), P.max_inner,
                                    breakdown);
        for (int i = threadIdx.x; i < n; i += 2 * BS) {
            const int j = i + BS;
            const double xi = V.x[S.o + i], di = (double)V.d32[S.o + i];
            double xj = 0.0, dj = 0.0;
            if (j < n) { xj = V.x[S.o + j]; dj = (double)V.d32[S.o + j]; }
            V.x[S.o + i] = fma(sc, di, xi);
            if (j < n) V.x[S.o + j] = fma(sc, dj, xj);
        }
        __syncthreads();
        ++outer_g;
    }
    if (threadIdx.x == 0) {
        const bool ok = (rr <= stop || bb == 0.0) && !breakdown;
        st[0] = breakdown ? LC_ERR_BREAKDOWN : (ok ? LC_OK : LC_ERR_NOT_CONVERGED);
        st[1] = K;
        st[2] = nzB;
        st[3] = it_l;
        st[4] = it_g;
        st[5] = outer_l;
        st[6] = outer_g;
        st[7] = outer_g == 0 ? 1 : 0;
        sd[0] = tau;
        sd[1] = bb > 0.0 ? sqrt(rr0 / bb) : 0.0;
        sd[2] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        sd[3] = sqrt(bb);
    }
    __syncthreads();
}

template <int BS>
__global__ void __launch_bounds__(BS) batched_kernel(BatchView V, BatchParams P) {
    __shared__ double red[128];
    __shared__ unsigned long long scan_sm[64];
    __shared__ int s_next;
    Blk<BS> blk{red};
    while (true) {
        if (threadIdx.x == 0) s_next = atomicAdd(V.next, 1);
        __syncthreads();
        const int k = s_next;
        __syncthreads();
        if (k >= V.nsys) break;
        solve_system<BS>(V, P, V.order[k], blk, scan_sm);
    }
}

__global__ void batch_f32_kernel(int64_t n, const double *D, const double *Tx, const double *Ty, float *D32,
                                 float *Tx32, float *Ty32, float *dinv32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        D32[i] = (float)D[i];
        Tx32[i] = (float)Tx[i];
        Ty32[i] = (float)Ty[i];
        dinv32[i] = 1.0f / (float)D[i];
    }
}

}  // namespace

namespace {
const void *batched_kernel_for(int block) {
    switch (block) {
        case 256: return (const void *)batched_kernel<256>;
        case 512: return (const void *)batched_kernel<512>;
        default: return (const void *)batched_kernel<1024>;
    }
}
}  // namespace

int batched_occupancy(int block) {
    int per = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_kernel_for(block), block, 0);
    return per < 1 ? 1 : per;
}

cudaError_t launch_batched(const void *launch_desc, int sms, cudaStream_t s) {
    const BatchLaunch &L = *static_cast<const BatchLaunch *>(launch_desc);
    int per = batched_occupancy(L.block);
    if (L.ctas_per_sm > 0 && L.ctas_per_sm < per) per = L.ctas_per_sm;
    int grid = sms * per;
    if (grid > L.v.nsys) grid = L.v.nsys;
    if (grid < 1) grid = 1;
    BatchView v = L.v;
    BatchParams prm = L.p;
    void *args[] = {&v, &prm};
    const cudaError_t e = cudaLaunchKernel(batched_kernel_for(L.block), dim3(grid), dim3(L.block), args, 0, s);
    note_launches(1);
    return e;
}

cudaError_t launch_batch_f32(int64_t n, const double *D, const double *Tx, const double *Ty, float *D32, float *Tx32,
                             float *Ty32, float *dinv32, cudaStream_t s) {
    batch_f32_kernel<<<152 * 8, 256, 0, s>>>(n, D, Tx, Ty, D32, Tx32, Ty32, dinv32);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace lc
