// lc_batched.cu -- many independent 2D systems, each solved by Alg 1 end to
// end, in ONE persistent launch (captured in a CUDA graph by lc_api.cu).
//
// Every system is solved by a team -- one CTA, or a thread-block cluster of
// 2, 4, 8 or 16 CTAs -- with team-level synchronisation
// only (systems are independent, so there is no grid-wide wait):
//   residual marking  r0 = b - A x0 in the canonical order, tau = beta max|r0|,
//                     mask = |r0| > tau, `layers` rounds of dilation  (Alg 3 variant)
//   extraction        packed-pair scan -> g2l, l2g, rowptr; B, rhs, xL0  (Eq. loc-equ)
//   local solve       iterative refinement: FP64 residual, FP32 Jacobi-CG on fl32(B)
//   assembly          x~ = x0 with x~[l2g] = xL                          (Eq. sol-assemble)
//   check + global    iterative refinement on the whole system from x~; returns at once
//                     if ||b - A x~|| <= tol ||b||                       (Alg 1 steps 8-11)
// The masks and subsystems are bit-identical to lc_mark_residual / lc_extract
// on the same system (same canonical orders; the threshold's max does not
// depend on the order); the solves reach the same FP64 relative residual.
//
// Work queues: the systems sorted by size, largest first.  With clusters the
// first `nbig` of them (at least big_cells cells) go to whole clusters -- the
// cluster's leader takes the next one and hands its index to the other CTAs
// through distributed shared memory -- and, once those are taken, every CTA
// takes the remaining systems one at a time on its own.  On a cluster a
// system's rows are split into contiguous ranges, one per CTA; a team sum is
// the CTAs' block sums pushed into every CTA's shared memory and added in
// rank order after a cluster barrier (the same total in every CTA); values
// that another CTA of the cluster wrote (neighbours across a range boundary)
// are read through L2.  A 512 x 512 system on one SM is what bounded the
// whole batch before (10 ms of a 21.8 ms batch).
#include <cooperative_groups.h>

#include "lc_internal.cuh"

namespace lc {

namespace {

namespace cg = cooperative_groups;

constexpr int kMaxTeam = 16;

// each CTA's receiving area for the team's exchanges: two alternating sets
// (a fast CTA may push into set k+1 while a slower one still reads set k,
// but not into set k+2 before every CTA passed exchange k+1's barrier)
struct TeamSm {
    double d[2][kMaxTeam][4];
    unsigned long long u[2][kMaxTeam];
};

// A team: one CTA (size 1) or the `size` CTAs of a cluster.  Every thread of
// every CTA of the team calls the same sequence of team operations.
template <int BS>
struct Team {
    int rank, size;
    double *red;                  // block scratch, >= 128 doubles
    unsigned long long *scan_sm;  // block scratch, >= 64 words
    TeamSm *ts;                   // this CTA's exchange area
    int buf;

    __device__ void sync() const {
        if (size > 1) cg::this_cluster().sync();
        else __syncthreads();
    }
    // thread 0's NV values into row `rank` of set `buf` of every CTA, then the
    // barrier; returns the set to read
    template <int NV>
    __device__ int push(const double (&v)[NV]) {
        if (threadIdx.x < 32) {
            double w[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) w[k] = __shfl_sync(kFull, v[k], 0);
            if ((int)threadIdx.x < size) {
                double *dst = cg::this_cluster().map_shared_rank(&ts->d[buf][rank][0], threadIdx.x);
#pragma unroll
                for (int k = 0; k < NV; ++k) dst[k] = w[k];
            }
        }
        cg::this_cluster().sync();
        const int b = buf;
        buf ^= 1;
        return b;
    }
    // team sums of NV FP64 values per thread (every thread gets the totals)
    template <int NV>
    __device__ void sum(double (&v)[NV]) {
        block_sum<NV, double>(v, red);
        if (size > 1) {
            const int b = push<NV>(v);
            if (threadIdx.x == 0)
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    double s = 0.0;
                    for (int c = 0; c < size; ++c) s += ts->d[b][c][k];
                    v[k] = s;
                }
        }
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k) red[96 + k] = v[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = red[96 + k];
        __syncthreads();
    }
    __device__ double sum1(double v) {
        double a[1] = {v};
        sum<1>(a);
        return a[0];
    }
    // team sums of two FP32 values per thread: FP32 block sums, added across
    // the team in FP64 (exact for two terms, rounded once per further term)
    __device__ void sum2f(float &u, float &v) {
        float a[2] = {u, v};
        block_sum<2, float>(a, reinterpret_cast<float *>(red));
        double t[2] = {(double)a[0], (double)a[1]};
        if (size > 1) {
            const int b = push<2>(t);
            if (threadIdx.x == 0)
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    double s = 0.0;
                    for (int c = 0; c < size; ++c) s += ts->d[b][c][k];
                    t[k] = s;
                }
        }
        if (threadIdx.x == 0) { red[96] = (double)(float)t[0]; red[97] = (double)(float)t[1]; }
        __syncthreads();
        u = (float)red[96];
        v = (float)red[97];
        __syncthreads();
    }
    // team maximum of a 64-bit key per thread
    __device__ unsigned long long max_u64(unsigned long long v) {
        v = block_max(v, scan_sm);
        if (size > 1) {
            if (threadIdx.x < 32) {
                const unsigned long long w = __shfl_sync(kFull, v, 0);
                if ((int)threadIdx.x < size)
                    *cg::this_cluster().map_shared_rank(&ts->u[buf][rank], threadIdx.x) = w;
            }
            cg::this_cluster().sync();
            if (threadIdx.x == 0) {
                unsigned long long m = 0;
                for (int c = 0; c < size; ++c) m = ts->u[buf][c] > m ? ts->u[buf][c] : m;
                v = m;
            }
            buf ^= 1;
        }
        if (threadIdx.x == 0) scan_sm[40] = v;
        __syncthreads();
        v = scan_sm[40];
        __syncthreads();
        return v;
    }
    // exclusive prefix over the team's ranks of one 64-bit total per CTA
    // (thread 0's `v`), and the team total; every thread gets both
    __device__ unsigned long long excl_scan_u64(unsigned long long v, unsigned long long &total) {
        unsigned long long pre = 0, tot = v;
        if (size > 1) {
            if (threadIdx.x < 32) {
                const unsigned long long w = __shfl_sync(kFull, v, 0);
                if ((int)threadIdx.x < size)
                    *cg::this_cluster().map_shared_rank(&ts->u[buf][rank], threadIdx.x) = w;
            }
            cg::this_cluster().sync();
            if (threadIdx.x == 0) {
                tot = 0;
                for (int c = 0; c < size; ++c) {
                    if (c == rank) pre = tot;
                    tot += ts->u[buf][c];
                }
            }
            buf ^= 1;
        }
        if (threadIdx.x == 0) { scan_sm[41] = pre; scan_sm[42] = tot; }
        __syncthreads();
        pre = scan_sm[41];
        total = scan_sm[42];
        __syncthreads();
        return pre;
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

// A value another CTA of the team wrote (a neighbour beyond this CTA's rows)
// is read through L2 (`other`); everything else, including the team's own
// rows, through L1 as usual.
template <bool TEAM, typename T>
__device__ __forceinline__ T ldn(const T *p, bool other) {
    if constexpr (TEAM) {
        if (other) return __ldcg(p);
    }
    return *p;
}

// one system -----------------------------------------------------------------

struct Sys {
    int nx, ny, n;
    int64_t o;     // cell offset
    int64_t oe;    // offset of B's entries (5 o)
    int64_t orp;   // offset of B's row pointers (o + s)
    int y0, y1;    // this CTA's grid rows
    int l0, l1;    // this CTA's rows of the subsystem
    int K;         // rows of the subsystem
};

// canonical residual of cell i (local index), FP64
template <bool TEAM>
__device__ __forceinline__ double res_row(const BatchView &V, const Sys &S, const double *x, int i) {
    const int ux = i % S.nx, uy = i / S.nx;
    const int64_t g = S.o + i;
    double r = V.b[g];
    if (uy > 0) r = __fma_rn(V.Ty[g - S.nx], ldn<TEAM>(x + g - S.nx, uy == S.y0), r);
    if (ux > 0) r = __fma_rn(V.Tx[g - 1], x[g - 1], r);
    r = __fma_rn(-V.D[g], x[g], r);
    if (ux + 1 < S.nx) r = __fma_rn(V.Tx[g], x[g + 1], r);
    if (uy + 1 < S.ny) r = __fma_rn(V.Ty[g], ldn<TEAM>(x + g + S.nx, uy + 1 == S.y1), r);
    return r;
}

// q = A32 p on the FP32 stencil (local index i)
template <bool TEAM>
__device__ __forceinline__ float spmv32(const BatchView &V, const Sys &S, const float *p, int i) {
    const int ux = i % S.nx, uy = i / S.nx;
    const int64_t g = S.o + i;
    float q = V.D32[g] * p[g];
    if (uy > 0) q = fmaf(-V.Ty32[g - S.nx], ldn<TEAM>(p + g - S.nx, uy == S.y0), q);
    if (ux > 0) q = fmaf(-V.Tx32[g - 1], p[g - 1], q);
    if (ux + 1 < S.nx) q = fmaf(-V.Tx32[g], p[g + 1], q);
    if (uy + 1 < S.ny) q = fmaf(-V.Ty32[g], ldn<TEAM>(p + g + S.nx, uy + 1 == S.y1), q);
    return q;
}

// Reduction asked of a sweep's inner solve: inner_tol, or -- when the outer
// test (rr <= stop) misses by less -- half of what is still missing.
__device__ __forceinline__ double sweep_tol(double inner_tol, double stop, double rr) {
    const double need = 0.5 * sqrt(stop / rr);
    return need > inner_tol ? need : inner_tol;
}

// FP32 Jacobi-CG on (A32 | B32) d = r32 from d = 0 over the unknowns
// [lo, hi) of this CTA (cells of the system, or rows of its subsystem, at
// `o`); stops when the residual fell by inner_tol or after max_inner
// iterations.  Returns iterations (the same in every CTA of the team).
// Each thread takes its unknowns two at a time (i, i + BS) and issues both
// unknowns' loads before either one's stores: a store whose value waits on
// a load would otherwise hold every later load back (the compiler cannot
// prove the arrays apart), one memory latency per unknown.  Sums keep the
// order i, i + BS, i + 2 BS, ... of a plain strided loop.  (Measured on the
// 512-system batch: one unknown per trip 28.3 ms, two 21.6 ms; generic
// loops over 2, 4 or 8 unknowns came out between 21.3 and 27.5 ms, and
// slower on the small multi-group systems.  Forming p = z + beta p_old
// inside the product at all five points, to save the separate p pass and
// one team sync per iteration, made it slower still: 20.7 -> 24.9 ms, and
// 0.87 -> 1.10 ms on the multi-group batch -- twice the neighbour loads.)
template <int BS, bool CSR, bool TEAM>
__device__ int inner_cg(const BatchView &V, const Sys &S, Team<BS> &tm, int lo, int hi, int64_t o, const float *dinv,
                        double inner_tol, int max_inner, int &breakdown) {
    float *r = V.r32 + o, *z = V.z32 + o, *p = V.p32 + o, *q = V.q32 + o, *d = V.d32 + o;
    auto aq = [&](int i) {   // (A p)_i or (B p)_i
        if (CSR) {
            float qi = 0.f;
            const int32_t e0 = V.rowptr[S.orp + i], e1 = ldn<TEAM>(V.rowptr + S.orp + i + 1, i + 1 == S.l1);
            for (int32_t e = e0; e < e1; ++e) {
                const int32_t c = LC_IDX(V.col[S.oe + e], S.K);
                qi = fmaf(V.val32[S.oe + e], ldn<TEAM>(p + c, c < S.l0 || c >= S.l1), qi);
            }
            return qi;
        } else {
            return spmv32<TEAM>(V, S, V.p32, i);
        }
    };
    float rz = 0.f, rr = 0.f;
    for (int i = lo + threadIdx.x; i < hi; i += 2 * BS) {
        const int j = i + BS;
        const bool two = j < hi;
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
    tm.sum2f(rz, rr);
    const float stop = (float)(inner_tol * inner_tol) * rr;
    int it = 0;
    while (it < max_inner && rr > stop) {
        float pq = 0.f;
        for (int i = lo + threadIdx.x; i < hi; i += 2 * BS) {
            const int j = i + BS;
            const bool two = j < hi;
            const float qi = aq(i), pi = p[i];
            float qj = 0.f, pj = 0.f;
            if (two) { qj = aq(j); pj = p[j]; }
            q[i] = qi;
            pq = fmaf(pi, qi, pq);
            if (two) { q[j] = qj; pq = fmaf(pj, qj, pq); }
        }
        float dummy = 0.f;
        tm.sum2f(pq, dummy);
        if (!(pq > 0.f) || !isfinite(pq)) { breakdown = 1; break; }
        const float alpha = rz / pq;
        float rz2 = 0.f, rr2 = 0.f;
        for (int i = lo + threadIdx.x; i < hi; i += 2 * BS) {
            const int j = i + BS;
            const bool two = j < hi;
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
        tm.sum2f(rz2, rr2);
        ++it;
        const float beta = rz2 / rz;
        rz = rz2;
        rr = rr2;
        for (int i = lo + threadIdx.x; i < hi; i += 2 * BS) {
            const int j = i + BS;
            const bool two = j < hi;
            const float pi = p[i], zi = z[i];
            float pj = 0.f, zj = 0.f;
            if (two) { pj = p[j]; zj = z[j]; }
            p[i] = fmaf(beta, pi, zi);
            if (two) p[j] = fmaf(beta, pj, zj);
        }
        tm.sync();   // the next product reads neighbours' p
    }
    return it;
}

// Alg 1 on system s by the team (this CTA: the rows of its range).
template <int BS, bool TEAM>
__device__ void solve_system(const BatchView &V, const BatchParams &P, int s, Team<BS> &tm) {
    Sys S;
    S.nx = V.nx[s];
    S.ny = V.ny[s];
    S.n = S.nx * S.ny;
    S.o = V.off[s];
    S.oe = 5 * S.o;
    S.orp = S.o + s;
    // this CTA's cells: a contiguous range of whole rows
    const int rows = (S.ny + tm.size - 1) / tm.size;
    S.y0 = min(S.ny, tm.rank * rows);
    S.y1 = min(S.ny, S.y0 + rows);
    S.l0 = S.l1 = S.K = 0;
    const int lo = S.y0 * S.nx, hi = S.y1 * S.nx;
    int32_t *st = V.stat_i + 8 * (int64_t)s;
    double *sd = V.stat_d + 4 * (int64_t)s;
    int breakdown = 0;

    // ---- residual marking (canonical residual, relative threshold, layers)
    unsigned long long mx = 0;
    for (int i = lo + threadIdx.x; i < hi; i += 2 * BS) {   // two cells at a time, loads before stores
        const int j = i + BS;
        const double ri = res_row<TEAM>(V, S, V.x, i);
        const double rj = j < hi ? res_row<TEAM>(V, S, V.x, j) : 0.0;
        V.r[S.o + i] = ri;
        unsigned long long a = maxable_bits(ri);
        mx = a > mx ? a : mx;
        if (j < hi) {
            V.r[S.o + j] = rj;
            a = maxable_bits(rj);
            mx = a > mx ? a : mx;
        }
    }
    mx = tm.max_u64(mx);
    const double tau = __dmul_rn(P.beta, __longlong_as_double((long long)mx));
    const unsigned long long tbits = abs_bits(tau);
    uint8_t *ma = V.m0 + S.o, *mb = V.m1 + S.o;
    for (int i = lo + threadIdx.x; i < hi; i += BS) ma[i] = (uint8_t)abs_gt(V.r[S.o + i], tbits);
    tm.sync();
    for (int l = 0; l < P.layers; ++l) {
        for (int i = lo + threadIdx.x; i < hi; i += BS) {
            const int ux = i % S.nx, uy = i / S.nx;
            uint8_t m = ma[i];
            if (!m) m = (uy > 0 && ldn<TEAM>(ma + i - S.nx, uy == S.y0)) | (ux > 0 && ma[i - 1]) |
                        (ux + 1 < S.nx && ma[i + 1]) | (uy + 1 < S.ny && ldn<TEAM>(ma + i + S.nx, uy + 1 == S.y1));
            mb[i] = m;
        }
        tm.sync();
        uint8_t *t = ma; ma = mb; mb = t;
    }

    // ---- compaction: one packed (cells, entries) scan over the cells in order
    auto packed = [&](int i) -> unsigned long long {
        if (i >= hi || !ma[i]) return 0ull;
        const int ux = i % S.nx, uy = i / S.nx;
        unsigned c = 1;
        if (uy > 0) c += ldn<TEAM>(ma + i - S.nx, uy == S.y0);
        if (ux > 0) c += ma[i - 1];
        if (ux + 1 < S.nx) c += ma[i + 1];
        if (uy + 1 < S.ny) c += ldn<TEAM>(ma + i + S.nx, uy + 1 == S.y1);
        return 1ull | ((unsigned long long)c << 32);
    };
    unsigned long long run = 0, total = 0;
    if (tm.size > 1) {   // the ranges before this CTA's: their totals
        unsigned long long mine = 0;
        for (int i = lo + threadIdx.x; i < hi; i += BS) mine += packed(i);
        unsigned long long blk;
        blk_scan(mine, tm.scan_sm, blk);
        run = tm.excl_scan_u64(blk, total);
    }
    int32_t *g2l = V.g2l + S.o, *l2g = V.l2g + S.o, *rp = V.rowptr + S.orp;
    const unsigned long long first = run;
    for (int base = lo; base < hi; base += BS) {
        const int i = base + threadIdx.x;
        const unsigned long long v = packed(i);
        unsigned long long tot;
        const unsigned long long pre = blk_scan(v, tm.scan_sm, tot) + run;
        if (i < hi) {
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
    if (tm.size == 1) total = run;
    const int K = (int)(total & 0xffffffffull);
    const int nzB = (int)(total >> 32);
    const int l0 = (int)(first & 0xffffffffull), l1 = (int)(run & 0xffffffffull);   // this CTA's local rows
    S.l0 = l0;
    S.l1 = l1;
    S.K = K;
    if (tm.rank == 0 && threadIdx.x == 0) rp[K] = nzB;
    tm.sync();

    // ---- gather B (FP64 and FP32 values), rhs (canonical order), xL0, 1/diag
    for (int l = l0 + threadIdx.x; l < l1; l += BS) {
        const int i = LC_IDX(l2g[l], S.n);
        const int ux = i % S.nx, uy = i / S.nx;
        const int64_t g = S.o + i;
        int32_t e = rp[l];
        double sacc = V.b[g];
        auto visit = [&](int j, double T) {
            const int jy = j / S.nx;
            const int32_t gj = ldn<TEAM>(g2l + j, jy < S.y0 || jy >= S.y1);
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
    tm.sync();

    // ---- local solve: iterative refinement on B (FP64 residual, FP32 CG)
    int it_l = 0, outer_l = 0;
    if (K > 0) {
        double bb = 0.0;
        for (int l = l0 + threadIdx.x; l < l1; l += BS) bb = fma(V.rhs[S.o + l], V.rhs[S.o + l], bb);
        bb = tm.sum1(bb);
        const double stop = (P.tol_local * P.tol_local) * bb;
        while (true) {
            double rr = 0.0;
            for (int l = l0 + threadIdx.x; l < l1; l += BS) {
                double a = 0.0;
                const int32_t e1 = ldn<TEAM>(rp + l + 1, l + 1 == S.l1);   // rp[K] is rank 0's
                for (int32_t e = rp[l]; e < e1; ++e) {
                    const int32_t c = LC_IDX(V.col[S.oe + e], S.K);
                    a = fma(V.val[S.oe + e], ldn<TEAM>(V.xl + S.o + c, c < S.l0 || c >= S.l1), a);
                }
                const double rl = V.rhs[S.o + l] - a;
                V.r[S.o + l] = rl;
                rr = fma(rl, rl, rr);
            }
            rr = tm.sum1(rr);
            if (rr <= stop || bb == 0.0 || outer_l >= P.max_outer) break;
            const double sc = sqrt(rr), inv = 1.0 / sc;
            for (int l = l0 + threadIdx.x; l < l1; l += BS) V.r32[S.o + l] = (float)(V.r[S.o + l] * inv);
            __syncthreads();
            it_l += inner_cg<BS, true, TEAM>(V, S, tm, l0, l1, S.o, V.dl32 + S.o, sweep_tol(P.inner_tol, stop, rr),
                                            P.max_inner, breakdown);
            for (int l = l0 + threadIdx.x; l < l1; l += BS)
                V.xl[S.o + l] = fma(sc, (double)V.d32[S.o + l], V.xl[S.o + l]);
            tm.sync();   // the next residual reads neighbours' xl
            ++outer_l;
            if (breakdown) break;
        }
    }
    // ---- assembly x~ = x0 with the local solution
    for (int l = l0 + threadIdx.x; l < l1; l += BS) V.x[S.o + LC_IDX(l2g[l], S.n)] = V.xl[S.o + l];
    tm.sync();

    // ---- check of x~ and global solve: iterative refinement on A
    int it_g = 0, outer_g = 0;
    double bb = 0.0, rr0 = 0.0, rr = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += BS) bb = fma(V.b[S.o + i], V.b[S.o + i], bb);
    bb = tm.sum1(bb);
    const double stop = (P.tol * P.tol) * bb;
    while (true) {
        rr = 0.0;
        for (int i = lo + threadIdx.x; i < hi; i += 2 * BS) {   // two cells at a time, loads before stores
            const int j = i + BS;
            const double ri = res_row<TEAM>(V, S, V.x, i);
            const double rj = j < hi ? res_row<TEAM>(V, S, V.x, j) : 0.0;
            V.r[S.o + i] = ri;
            rr = fma(ri, ri, rr);
            if (j < hi) {
                V.r[S.o + j] = rj;
                rr = fma(rj, rj, rr);
            }
        }
        rr = tm.sum1(rr);
        if (outer_g == 0) rr0 = rr;
        if (rr <= stop || bb == 0.0 || outer_g >= P.max_outer || breakdown) break;
        const double sc = sqrt(rr), inv = 1.0 / sc;
        for (int i = lo + threadIdx.x; i < hi; i += 2 * BS) {
            const int j = i + BS;
            const double ri = V.r[S.o + i], rj = j < hi ? V.r[S.o + j] : 0.0;
            V.r32[S.o + i] = (float)(ri * inv);
            if (j < hi) V.r32[S.o + j] = (float)(rj * inv);
        }
        __syncthreads();
        it_g += inner_cg<BS, false, TEAM>(V, S, tm, lo, hi, S.o, V.dinv32 + S.o, sweep_tol(P.inner_tol, stop, rr),
                                         P.max_inner, breakdown);
        for (int i = lo + threadIdx.x; i < hi; i += 2 * BS) {
            const int j = i + BS;
            const double xi = V.x[S.o + i], di = (double)V.d32[S.o + i];
            double xj = 0.0, dj = 0.0;
            if (j < hi) { xj = V.x[S.o + j]; dj = (double)V.d32[S.o + j]; }
            V.x[S.o + i] = fma(sc, di, xi);
            if (j < hi) V.x[S.o + j] = fma(sc, dj, xj);
        }
        tm.sync();   // the next residual reads neighbours' x
        ++outer_g;
    }
    if (tm.rank == 0 && threadIdx.x == 0) {
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

// C = 1: every CTA takes systems on its own.  C > 1 (launched as clusters of
// C CTAs): first the nbig largest systems, one per cluster, then the rest one
// per CTA.
template <int BS, int C>
__global__ void __launch_bounds__(BS) batched_kernel(BatchView V, BatchParams P) {
    __shared__ double red[128];
    __shared__ unsigned long long scan_sm[64];
    __shared__ TeamSm ts;
    __shared__ int s_next;
    if constexpr (C > 1) {
        cg::cluster_group cl = cg::this_cluster();
        Team<BS> tm{(int)cl.block_rank(), C, red, scan_sm, &ts, 0};
        while (true) {
            if (tm.rank == 0 && threadIdx.x == 0) {
                const int k = atomicAdd(V.next, 1);
                for (int c = 0; c < C; ++c) *cl.map_shared_rank(&s_next, c) = k;
            }
            cl.sync();
            const int k = s_next;
            cl.sync();   // every CTA has read s_next before the leader writes it again
            if (k >= V.nbig) break;
            solve_system<BS, true>(V, P, V.order[k], tm);
        }
    }
    Team<BS> solo{0, 1, red, scan_sm, &ts, 0};
    while (true) {
        if (threadIdx.x == 0) s_next = atomicAdd(V.next + 1, 1);
        __syncthreads();
        const int k = s_next;
        __syncthreads();
        if (k >= V.nsys - V.nbig) break;
        solve_system<BS, false>(V, P, V.order[V.nbig + k], solo);
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

template <int C>
const void *kernel_c(int block) {
    switch (block) {
        case 256: return (const void *)batched_kernel<256, C>;
        case 512: return (const void *)batched_kernel<512, C>;
        default: return (const void *)batched_kernel<1024, C>;
    }
}

const void *batched_kernel_for(int block, int cluster) {
    switch (cluster) {
        case 2: return kernel_c<2>(block);
        case 4: return kernel_c<4>(block);
        case 8: return kernel_c<8>(block);
        case 16: return kernel_c<16>(block);
        default: return kernel_c<1>(block);
    }
}

}  // namespace

int batched_occupancy(int block) {
    int per = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_kernel_for(block, 1), block, 0);
    return per < 1 ? 1 : per;
}

cudaError_t launch_batched(const void *launch_desc, int sms, cudaStream_t s) {
    const BatchLaunch &L = *static_cast<const BatchLaunch *>(launch_desc);
    BatchView v = L.v;
    BatchParams prm = L.p;
    void *args[] = {&v, &prm};
    const int C = L.cluster;
    int per = batched_occupancy(L.block);
    if (L.ctas_per_sm > 0 && L.ctas_per_sm < per) per = L.ctas_per_sm;
    if (C <= 1 || v.nbig == 0) {
        v.nbig = 0;
        int grid = sms * per;
        if (grid > v.nsys) grid = v.nsys;
        if (grid < 1) grid = 1;
        const cudaError_t e = cudaLaunchKernel(batched_kernel_for(L.block, 1), dim3(grid), dim3(L.block), args, 0, s);
        note_launches(1);
        return e;
    }
    const void *k = batched_kernel_for(L.block, C);
    if (C > 8) {   // 16 CTAs per cluster is beyond the portable size
        const cudaError_t ea = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (ea != cudaSuccess) return ea;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(L.block);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // as many clusters as fit at once (a persistent grid: the queues hand out the work)
    cfg.gridDim = dim3(sms * per / C * C);
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    const int per_cap = sms * per / C;   // ctas_per_sm limits the clusters too
    if (nclusters > per_cap && per_cap >= 1) nclusters = per_cap;
    cfg.gridDim = dim3(nclusters * C);
    e = cudaLaunchKernelExC(&cfg, k, args);
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
