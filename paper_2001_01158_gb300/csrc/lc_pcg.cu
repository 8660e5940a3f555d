// lc_pcg.cu -- Jacobi-preconditioned conjugate gradients as ONE persistent
// cooperative kernel per solve (the Krylov solver of Alg 1, steps 5 and 11).
//
// Per iteration two grid-wide phases, each closed by a bounded grid barrier
// and a deterministic fixed-slot reduction (every block sums the same block
// partials in the same order, so every block takes the same decisions):
//
//   phase A  p = z + beta p_old          (computed where it is needed, halos
//            q = A p, partial p.q          included, so no extra barrier)
//            store p (ping-pong buffer) and q
//   phase B  alpha = rz / pq; x += alpha p; r -= alpha q; z = dinv r;
//            partials r.z and r.r
//
// z is stored so that phase A reads one vector where it would read r and
// dinv; the stopping test ||r||^2 <= tol^2 ||b||^2 is taken on the recurrence
// residual, confirmed with the true residual b - A x, and the iteration
// restarts from the true residual when that misses (at most max_restarts).
// The test on the starting iterate happens in the set-up phase: a converged
// start (Alg 1 step 8, the local solution x~ already good enough) costs one
// residual pass and no iteration.
//
// Data movement per cell and iteration (2D, FP64): phase A reads z, p_old,
// D, Tx, Ty and writes p, q (56 B); phase B reads x, p, r, q, dinv and
// writes x, r, z (64 B): 120 B.  Structured operators march a column strip
// (2D) or an xy tile (3D) through the grid so that every p is computed once
// plus a thin halo; CSR rows recompute the p of their columns.
#include "lc_internal.cuh"

namespace lc {

namespace {

constexpr int kPcgThreads = 256;
constexpr int kStripRows = 16;     // 2D: rows per unit
constexpr int kTileX = 32, kTileY = 8, kTileZ = 16;   // 3D unit

struct Bufs {
    const double *b;
    double *x, *r, *z, *q;
    double *p0, *p1;
    const double *dinv;
    double *part;          // [6][kMaxGrid]
};

// -------------------------------------------------------------- operators
//
// Every operator provides, for the calling block:
//   setup_block     r = b - A x, z = dinv r over its cells; sums b.b, r.z, r.r
//   phaseA_block    p = z + beta p_old, q = A p over its cells; sums p.q
//   each_cell(f)    f(i) for its cells (phase B), in the same cell-to-thread
//                   mapping as phase A, so the p and q a thread stored are
//                   the ones it reads back.

// 2D: the grid is cut into column strips of kPcgThreads cells (one thread
// per column); the strip-major list of (strip, row) pairs is split evenly
// into contiguous ranges, one per block, and a block marches down its rows.
// p of the row above and below lives in registers, the two x-neighbours come
// from a shared-memory row (double-buffered: one barrier per row).
struct Op2D {
    Stencil s;
    __device__ __forceinline__ int strips() const { return (s.nx + kPcgThreads - 1) / kPcgThreads; }
    template <class F>
    __device__ __forceinline__ void each_segment(F f) const {
        const int64_t rs = (int64_t)strips() * s.ny;
        const int64_t lo = rs * blockIdx.x / gridDim.x, hi = rs * (blockIdx.x + 1) / gridDim.x;
        if (lo >= hi) return;
        const int st0 = (int)(lo / s.ny), st1 = (int)((hi - 1) / s.ny);
        for (int st = st0; st <= st1; ++st) {
            const int y0 = st == st0 ? (int)(lo % s.ny) : 0;
            const int y1 = st == st1 ? (int)((hi - 1) % s.ny) + 1 : s.ny;
            f(st * kPcgThreads, y0, y1);
        }
    }
    __device__ void setup_block(const Bufs &B, double &bb, double &rz, double &rr) const {
        each_segment([&](int x0, int y0, int y1) {
            const int xx = x0 + threadIdx.x;
            if (xx >= s.nx) return;
            for (int y = y0; y < y1; ++y) {
                const int64_t i = (int64_t)y * s.nx + xx;
                double ax = s.D[i] * ldcg(B.x + i);
                if (y > 0) ax = fma(-s.Ty[i - s.nx], ldcg(B.x + i - s.nx), ax);
                if (xx > 0) ax = fma(-s.Tx[i - 1], ldcg(B.x + i - 1), ax);
                if (xx + 1 < s.nx) ax = fma(-s.Tx[i], ldcg(B.x + i + 1), ax);
                if (y + 1 < s.ny) ax = fma(-s.Ty[i], ldcg(B.x + i + s.nx), ax);
                const double bi = B.b[i];
                const double ri = bi - ax;
                const double zi = s.dinv[i] * ri;
                B.r[i] = ri;
                B.z[i] = zi;
                bb = fma(bi, bi, bb);
                rz = fma(ri, zi, rz);
                rr = fma(ri, ri, rr);
            }
        });
    }
    __device__ __forceinline__ double pnew(const Bufs &B, const double *pold, bool first, double beta,
                                           int64_t i) const {
        const double zi = ldcg(B.z + i);
        return first ? zi : fma(beta, ldcg(pold + i), zi);
    }
    __device__ void phaseA_block(const Bufs &B, const double *pold, double *pout, bool first, double beta,
                                 double &pq, double *srow) const {
        each_segment([&](int x0, int y0, int y1) {
            const int xx = x0 + threadIdx.x;
            const bool act = xx < s.nx;
            const bool hw = threadIdx.x == 0 && x0 > 0;
            const bool he = threadIdx.x == kPcgThreads - 1 && x0 + kPcgThreads < s.nx;
            double pm = 0.0, pc = 0.0, tym = 0.0;
            if (act) {
                const int64_t i0 = (int64_t)y0 * s.nx + xx;
                pc = pnew(B, pold, first, beta, i0);
                if (y0 > 0) { pm = pnew(B, pold, first, beta, i0 - s.nx); tym = s.Ty[i0 - s.nx]; }
            }
            for (int y = y0; y < y1; ++y) {
                const int64_t i = (int64_t)y * s.nx + xx;
                // every load of this row first, then one barrier
                double pn = 0.0, d = 0.0, txw = 0.0, txe = 0.0, typ = 0.0, halo = 0.0;
                if (act) {
                    if (y + 1 < s.ny) { pn = pnew(B, pold, first, beta, i + s.nx); typ = s.Ty[i]; }
                    d = s.D[i];
                    if (xx > 0) txw = s.Tx[i - 1];
                    if (xx + 1 < s.nx) txe = s.Tx[i];
                }
                if (hw) halo = pnew(B, pold, first, beta, (int64_t)y * s.nx + x0 - 1);
                if (he) halo = pnew(B, pold, first, beta, (int64_t)y * s.nx + x0 + kPcgThreads);
                double *buf = srow + (y & 1) * (kPcgThreads + 2);
                buf[threadIdx.x + 1] = pc;
                if (threadIdx.x == 0) buf[0] = halo;
                if (threadIdx.x == kPcgThreads - 1) buf[kPcgThreads + 1] = halo;
                __syncthreads();
                if (act) {
                    double qi = d * pc;
                    qi = fma(-tym, pm, qi);
                    qi = fma(-txw, buf[threadIdx.x], qi);
                    qi = fma(-txe, buf[threadIdx.x + 2], qi);
                    qi = fma(-typ, pn, qi);
                    pout[i] = pc;
                    B.q[i] = qi;
                    pq = fma(pc, qi, pq);
                }
                tym = typ;
                pm = pc;
                pc = pn;
            }
            __syncthreads();
        });
    }
    template <class F>
    __device__ __forceinline__ void each_cell(F f) const {
        each_segment([&](int x0, int y0, int y1) {
            const int xx = x0 + threadIdx.x;
            if (xx >= s.nx) return;
#pragma unroll 4
            for (int y = y0; y < y1; ++y) f((int64_t)y * s.nx + xx);
        });
    }
    static constexpr int kSmem = 2 * (kPcgThreads + 2);
    __device__ void resolve() {}
};

// 2D, warp-independent: the grid is cut into column strips of 32*CPL cells,
// one lane owning CPL adjacent columns (CPL = 2 when nx is even, so that
// rows start 16-byte aligned and loads/stores are double2).  The strip-major
// list of (strip, row) items is split evenly over all warps of the grid and
// every warp marches down its own rows: p of the rows above and below in
// registers, x-neighbours through warp shuffles, the one-cell halo at either
// end of the strip recomputed by lanes 0 and 31.  No block barrier, no shared
// memory.
template <int CPL>
struct Op2DW {
    Stencil s;
    static constexpr int kSW = 32 * CPL;
    __device__ __forceinline__ int strips() const { return (s.nx + kSW - 1) / kSW; }
    template <class F>
    __device__ __forceinline__ void each_segment(F f) const {
        const int wpb = blockDim.x >> 5;
        const int64_t gw = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
        const int64_t nw = (int64_t)gridDim.x * wpb;
        const int64_t items = (int64_t)strips() * s.ny;
        const int64_t lo = items * gw / nw, hi = items * (gw + 1) / nw;
        if (lo >= hi) return;
        const int st0 = (int)(lo / s.ny), st1 = (int)((hi - 1) / s.ny);
        for (int st = st0; st <= st1; ++st) {
            const int y0 = st == st0 ? (int)(lo % s.ny) : 0;
            const int y1 = st == st1 ? (int)((hi - 1) % s.ny) + 1 : s.ny;
            f(st * kSW, y0, y1);
        }
    }
    __device__ __forceinline__ double pnew1(const Bufs &B, const double *pold, bool first, double beta,
                                            int64_t i) const {
        const double zi = ldcg(B.z + i);
        return first ? zi : fma(beta, ldcg(pold + i), zi);
    }
    // p of the lane's CPL cells starting at i (i even when CPL == 2)
    __device__ __forceinline__ void pnew(const Bufs &B, const double *pold, bool first, double beta, int64_t i,
                                        double (&p)[CPL]) const {
        if (CPL == 2) {
            const double2 z2 = ldcg(reinterpret_cast<const double2 *>(B.z + i));
            if (first) { p[0] = z2.x; p[CPL - 1] = z2.y; }
            else {
                const double2 o2 = ldcg(reinterpret_cast<const double2 *>(pold + i));
                p[0] = fma(beta, o2.x, z2.x);
                p[CPL - 1] = fma(beta, o2.y, z2.y);
            }
        } else {
            p[0] = pnew1(B, pold, first, beta, i);
        }
    }
    __device__ __forceinline__ void load2(const double *a, int64_t i, double (&v)[CPL]) const {
        if (CPL == 2) {
            const double2 t = *reinterpret_cast<const double2 *>(a + i);
            v[0] = t.x; v[CPL - 1] = t.y;
        } else {
            v[0] = a[i];
        }
    }
    __device__ void setup_block(const Bufs &B, double &bb, double &rz, double &rr) const {
        const int lane = threadIdx.x & 31;
        each_segment([&](int x0, int y0, int y1) {
            for (int y = y0; y < y1; ++y) {
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const int xx = x0 + CPL * lane + k;
                    if (xx >= s.nx) continue;
                    const int64_t i = (int64_t)y * s.nx + xx;
                    double ax = s.D[i] * ldcg(B.x + i);
                    if (y > 0) ax = fma(-s.Ty[i - s.nx], ldcg(B.x + i - s.nx), ax);
                    if (xx > 0) ax = fma(-s.Tx[i - 1], ldcg(B.x + i - 1), ax);
                    if (xx + 1 < s.nx) ax = fma(-s.Tx[i], ldcg(B.x + i + 1), ax);
                    if (y + 1 < s.ny) ax = fma(-s.Ty[i], ldcg(B.x + i + s.nx), ax);
                    const double bi = B.b[i];
                    const double ri = bi - ax;
                    const double zi = s.dinv[i] * ri;
                    B.r[i] = ri;
                    B.z[i] = zi;
                    bb = fma(bi, bi, bb);
                    rz = fma(ri, zi, rz);
                    rr = fma(ri, ri, rr);
                }
            }
        });
    }
    __device__ void phaseA_block(const Bufs &B, const double *pold, double *pout, bool first, double beta,
                                 double &pq, double *) const {
        const int lane = threadIdx.x & 31;
        each_segment([&](int x0, int y0, int y1) {
            const int xa = x0 + CPL * lane;          // first column of this lane
            const bool act = xa < s.nx;               // CPL == 2: nx even, so xa+1 < nx too
            // halo column of the strip handled by lane 0 (west) / lane 31 (east)
            const int hx = lane == 0 ? x0 - 1 : x0 + kSW;
            const bool hact = (lane == 0 && x0 > 0) || (lane == 31 && x0 + kSW < s.nx);
            double pm[CPL], pc[CPL], pn[CPL], tym[CPL];
#pragma unroll
            for (int k = 0; k < CPL; ++k) { pm[k] = 0.0; pc[k] = 0.0; tym[k] = 0.0; }
            if (act) {
                const int64_t i0 = (int64_t)y0 * s.nx + xa;
                pnew(B, pold, first, beta, i0, pc);
                if (y0 > 0) {
                    pnew(B, pold, first, beta, i0 - s.nx, pm);
                    load2(s.Ty, i0 - s.nx, tym);
                }
            }
            for (int y = y0; y < y1; ++y) {
                const int64_t i = (int64_t)y * s.nx + xa;
                double d[CPL], tx[CPL], typ[CPL];
                double txw0 = 0.0, ph = 0.0;
#pragma unroll
                for (int k = 0; k < CPL; ++k) { pn[k] = 0.0; d[k] = 0.0; tx[k] = 0.0; typ[k] = 0.0; }
                if (act) {
                    if (y + 1 < s.ny) { pnew(B, pold, first, beta, i + s.nx, pn); load2(s.Ty, i, typ); }
                    load2(s.D, i, d);
                    load2(s.Tx, i, tx);
                    if (lane == 0 && x0 > 0) txw0 = s.Tx[i - 1];
                }
                if (hact) ph = pnew1(B, pold, first, beta, (int64_t)y * s.nx + hx);
                // face conductances to the west / east of each cell
                const double tx_last_up = __shfl_up_sync(kFull, tx[CPL - 1], 1);
                const double pc_last_up = __shfl_up_sync(kFull, pc[CPL - 1], 1);
                const double pc_first_dn = __shfl_down_sync(kFull, pc[0], 1);
                if (!act) continue;
                double txw[CPL], txe[CPL], pw[CPL], pe[CPL];
                txw[0] = lane == 0 ? txw0 : tx_last_up;
                pw[0] = lane == 0 ? ph : pc_last_up;
#pragma unroll
                for (int k = 1; k < CPL; ++k) { txw[k] = tx[k - 1]; pw[k] = pc[k - 1]; }
#pragma unroll
                for (int k = 0; k < CPL - 1; ++k) { txe[k] = tx[k]; pe[k] = pc[k + 1]; }
                const bool last_col = xa + CPL >= s.nx;   // the lane's last cell is the grid's last column
                txe[CPL - 1] = last_col ? 0.0 : tx[CPL - 1];
                pe[CPL - 1] = lane == 31 ? ph : pc_first_dn;
                double q[CPL];
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    double qi = d[k] * pc[k];
                    qi = fma(-tym[k], pm[k], qi);
                    qi = fma(-txw[k], pw[k], qi);
                    qi = fma(-txe[k], pe[k], qi);
                    qi = fma(-typ[k], pn[k], qi);
                    q[k] = qi;
                    pq = fma(pc[k], qi, pq);
                }
                if (CPL == 2) {
                    *reinterpret_cast<double2 *>(pout + i) = make_double2(pc[0], pc[CPL - 1]);
                    *reinterpret_cast<double2 *>(B.q + i) = make_double2(q[0], q[CPL - 1]);
                } else {
                    pout[i] = pc[0];
                    B.q[i] = q[0];
                }
#pragma unroll
                for (int k = 0; k < CPL; ++k) { tym[k] = typ[k]; pm[k] = pc[k]; pc[k] = pn[k]; }
            }
        });
    }
    template <class F>
    __device__ __forceinline__ void each_cell(F f) const {
        const int lane = threadIdx.x & 31;
        each_segment([&](int x0, int y0, int y1) {
            const int xa = x0 + CPL * lane;
            if (xa >= s.nx) return;
#pragma unroll 2
            for (int y = y0; y < y1; ++y)
#pragma unroll
                for (int k = 0; k < CPL; ++k) f((int64_t)y * s.nx + xa + k);
        });
    }
    static constexpr int kSmem = 1;
    __device__ void resolve() {}
};

struct Op3D {
    Stencil s;
    __device__ int64_t units() const {
        const int64_t tx = (s.nx + kTileX - 1) / kTileX, ty = (s.ny + kTileY - 1) / kTileY;
        const int64_t tz = (s.nz + kTileZ - 1) / kTileZ;
        return tx * ty * tz;
    }
    __device__ void origin(int64_t u, int &x0, int &y0, int &z0) const {
        const int64_t tx = (s.nx + kTileX - 1) / kTileX, ty = (s.ny + kTileY - 1) / kTileY;
        x0 = (int)(u % tx) * kTileX;
        y0 = (int)((u / tx) % ty) * kTileY;
        z0 = (int)(u / (tx * ty)) * kTileZ;
    }
    template <class F>
    __device__ void for_cells(int64_t u, F f) const {
        int x0, y0, z0;
        origin(u, x0, y0, z0);
        const int xx = x0 + (threadIdx.x % kTileX), yy = y0 + (threadIdx.x / kTileX);
        if (xx >= s.nx || yy >= s.ny) return;
        const int z1 = min(z0 + kTileZ, s.nz);
        const int64_t sxy = (int64_t)s.nx * s.ny;
        for (int z = z0; z < z1; ++z) f(xx + (int64_t)s.nx * yy + sxy * z);
    }
    template <class F>
    __device__ __forceinline__ void each_cell(F f) const {
        const int64_t nu = units();
        for (int64_t u = blockIdx.x; u < nu; u += gridDim.x) for_cells(u, f);
    }
    __device__ void setup_block(const Bufs &B, double &bb, double &rz, double &rr) const {
        const int64_t sxy = (int64_t)s.nx * s.ny;
        each_cell([&](int64_t i) {
            const int xx = (int)(i % s.nx), yy = (int)((i / s.nx) % s.ny), zz = (int)(i / sxy);
            double ax = s.D[i] * ldcg(B.x + i);
            if (zz > 0) ax = fma(-s.Tz[i - sxy], ldcg(B.x + i - sxy), ax);
            if (yy > 0) ax = fma(-s.Ty[i - s.nx], ldcg(B.x + i - s.nx), ax);
            if (xx > 0) ax = fma(-s.Tx[i - 1], ldcg(B.x + i - 1), ax);
            if (xx + 1 < s.nx) ax = fma(-s.Tx[i], ldcg(B.x + i + 1), ax);
            if (yy + 1 < s.ny) ax = fma(-s.Ty[i], ldcg(B.x + i + s.nx), ax);
            if (zz + 1 < s.nz) ax = fma(-s.Tz[i], ldcg(B.x + i + sxy), ax);
            const double bi = B.b[i];
            const double ri = bi - ax;
            const double zi = s.dinv[i] * ri;
            B.r[i] = ri;
            B.z[i] = zi;
            bb = fma(bi, bi, bb);
            rz = fma(ri, zi, rz);
            rr = fma(ri, ri, rr);
        });
    }
    // p of plane z (tile + 1-cell xy halo) into a (kTileY+2) x (kTileX+2) buffer
    __device__ void build_plane(const Bufs &B, const double *pold, bool first, double beta, int x0, int y0, int z,
                                double *pl) const {
        const int64_t sxy = (int64_t)s.nx * s.ny;
        constexpr int ex = kTileX + 2, ey = kTileY + 2;
        for (int k = threadIdx.x; k < ex * ey; k += kPcgThreads) {
            const int gx = x0 - 1 + (k % ex), gy = y0 - 1 + (k / ex);
            double v = 0.0;
            if (z >= 0 && z < s.nz && gx >= 0 && gx < s.nx && gy >= 0 && gy < s.ny) {
                const int64_t i = gx + (int64_t)s.nx * gy + sxy * z;
                const double zi = ldcg(B.z + i);
                v = first ? zi : fma(beta, ldcg(pold + i), zi);
            }
            pl[k] = v;
        }
    }
    __device__ void phaseA_block(const Bufs &B, const double *pold, double *pout, bool first, double beta,
                                 double &pq, double *sm) const {
        const int64_t nu = units();
        for (int64_t u = blockIdx.x; u < nu; u += gridDim.x) phaseA_unit(u, B, pold, pout, first, beta, pq, sm);
    }
    __device__ void phaseA_unit(int64_t u, const Bufs &B, const double *pold, double *pout, bool first, double beta,
                                double &pq, double *sm) const {
        constexpr int ex = kTileX + 2, ey = kTileY + 2, pls = ex * ey;
        int x0, y0, z0;
        origin(u, x0, y0, z0);
        const int lx = threadIdx.x % kTileX, ly = threadIdx.x / kTileX;
        const int xx = x0 + lx, yy = y0 + ly;
        const bool act = xx < s.nx && yy < s.ny;
        const int z1 = min(z0 + kTileZ, s.nz);
        const int64_t sxy = (int64_t)s.nx * s.ny;
        // planes z0-1 and z0 first
        build_plane(B, pold, first, beta, x0, y0, z0 - 1, sm + ((z0 + 3) & 3) * pls);
        build_plane(B, pold, first, beta, x0, y0, z0, sm + (z0 & 3) * pls);
        const int c = (ly + 1) * ex + (lx + 1);
        for (int z = z0; z < z1; ++z) {
            build_plane(B, pold, first, beta, x0, y0, z + 1, sm + ((z + 1) & 3) * pls);
            __syncthreads();
            if (act) {
                const double *pc = sm + (z & 3) * pls;
                const double pmz = sm[((z + 3) & 3) * pls + c];
                const double ppz = sm[((z + 1) & 3) * pls + c];
                const int64_t i = xx + (int64_t)s.nx * yy + sxy * z;
                const double p0 = pc[c];
                double qi = s.D[i] * p0;
                if (z > 0) qi = fma(-s.Tz[i - sxy], pmz, qi);
                if (yy > 0) qi = fma(-s.Ty[i - s.nx], pc[c - ex], qi);
                if (xx > 0) qi = fma(-s.Tx[i - 1], pc[c - 1], qi);
                if (xx + 1 < s.nx) qi = fma(-s.Tx[i], pc[c + 1], qi);
                if (yy + 1 < s.ny) qi = fma(-s.Ty[i], pc[c + ex], qi);
                if (z + 1 < s.nz) qi = fma(-s.Tz[i], ppz, qi);
                pout[i] = p0;
                B.q[i] = qi;
                pq = fma(p0, qi, pq);
            }
        }
        __syncthreads();
    }
    static constexpr int kSmem = 4 * (kTileX + 2) * (kTileY + 2);
    __device__ void resolve() {}
};

struct OpCsr {
    Csr c;
    int32_t n;   // resolved at kernel start (device-side count of an extracted subsystem)
    __device__ void resolve() { if (c.n_dev) n = *c.n_dev; }
    __device__ int64_t units() const { return (n + kPcgThreads - 1) / kPcgThreads; }
    template <class F>
    __device__ __forceinline__ void each_cell(F f) const {
        for (int64_t i = blockIdx.x * (int64_t)kPcgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kPcgThreads)
            f(i);
    }
    __device__ void setup_block(const Bufs &B, double &bb, double &rz, double &rr) const {
        each_cell([&](int64_t i) {
            double ax = 0.0;
            const int32_t e1 = c.rp[i + 1];
            for (int32_t e = c.rp[i]; e < e1; ++e) ax = fma(c.av[e], ldcg(B.x + c.ci[e]), ax);
            const double bi = B.b[i];
            const double ri = bi - ax;
            const double zi = B.dinv[i] * ri;
            B.r[i] = ri;
            B.z[i] = zi;
            bb = fma(bi, bi, bb);
            rz = fma(ri, zi, rz);
            rr = fma(ri, ri, rr);
        });
    }
    __device__ void phaseA_block(const Bufs &B, const double *pold, double *pout, bool first, double beta,
                                 double &pq, double *) const {
        each_cell([&](int64_t i) {
            double qi = 0.0, pi = 0.0;
            const int32_t e1 = c.rp[i + 1];
            for (int32_t e = c.rp[i]; e < e1; ++e) {
                const int32_t j = c.ci[e];
                const double zj = ldcg(B.z + j);
                const double pj = first ? zj : fma(beta, ldcg(pold + j), zj);
                if (j == i) pi = pj;
                qi = fma(c.av[e], pj, qi);
            }
            pout[i] = pi;
            B.q[i] = qi;
            pq = fma(pi, qi, pq);
        });
    }
    static constexpr int kSmem = 1;
};

// -------------------------------------------------------------- kernel

// Deterministic grid-wide sum of slot `k` of the block partials: every block
// computes the same value in the same order.
__device__ __forceinline__ double grid_reduce(const double *part, int k, unsigned nb, double *bcast) {
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (unsigned b = threadIdx.x; b < nb; b += 32) v += ldcg(part + (size_t)k * kMaxGrid + b);
        v = warp_sum(v);
        if (threadIdx.x == 0) *bcast = v;
    }
    __syncthreads();
    const double r = *bcast;
    __syncthreads();
    return r;
}

template <class OP>
__device__ bool setup_phase(const OP &op, const Bufs &B, double *red, double &bb, double &rz, double &rr,
                            Ctrl *ctrl) {
    double acc[3] = {0.0, 0.0, 0.0};
    op.setup_block(B, acc[0], acc[1], acc[2]);
    block_sum<3>(acc, red);
    if (threadIdx.x == 0) {
        B.part[0 * kMaxGrid + blockIdx.x] = acc[0];
        B.part[1 * kMaxGrid + blockIdx.x] = acc[1];
        B.part[2 * kMaxGrid + blockIdx.x] = acc[2];
    }
    if (!grid_sync(ctrl, gridDim.x)) return false;
    bb = grid_reduce(B.part, 0, gridDim.x, red + 96);
    rz = grid_reduce(B.part, 1, gridDim.x, red + 96);
    rr = grid_reduce(B.part, 2, gridDim.x, red + 96);
    return true;
}

template <class OP, int MINB>
__global__ void __launch_bounds__(kPcgThreads, MINB) pcg_kernel(OP op, Bufs B, double tol, int maxit, int max_restarts,
                                                          Ctrl *ctrl) {
    __shared__ double red[128];
    __shared__ double sm[OP::kSmem];
    op.resolve();
    double bb, rz, rr;
    if (!setup_phase(op, B, red, bb, rz, rr, ctrl)) return;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const double stop = (tol * tol) * bb;
    if (lead) {
        ctrl->bnorm2 = bb;
        ctrl->relres0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        ctrl->iters = 0;
        ctrl->restarts = 0;
    }
    if (bb == 0.0) {   // A x = 0: x = 0
        op.each_cell([&](int64_t i) { B.x[i] = 0.0; });
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = 0.0; }
        return;
    }
    if (rr <= stop) {
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = sqrt(rr / bb); }
        return;
    }
    int it = 0, restarts = 0, pin = 0;
    bool first = true;
    double beta = 0.0;
    int result = 0;   // 1 converged, 0 not converged, -1 breakdown
    while (true) {
        // ---- phase A
        double pq = 0.0;
        const double *pold = pin ? B.p1 : B.p0;
        double *pout = pin ? B.p0 : B.p1;
        op.phaseA_block(B, pold, pout, first, beta, pq, sm);
        {
            double a1[1] = {pq};
            block_sum<1>(a1, red);
            if (threadIdx.x == 0) B.part[3 * kMaxGrid + blockIdx.x] = a1[0];
        }
        if (!grid_sync(ctrl, gridDim.x)) return;
        pq = grid_reduce(B.part, 3, gridDim.x, red + 96);
        if (!(pq > 0.0) || !isfinite(pq)) { result = -1; break; }
        const double alpha = rz / pq;
        pin ^= 1;
        const double *p = pout;
        // ---- phase B
        double acc[2] = {0.0, 0.0};
        op.each_cell([&](int64_t i) {
            const double pi = p[i], qi = B.q[i];
            B.x[i] = fma(alpha, pi, B.x[i]);
            const double ri = fma(-alpha, qi, B.r[i]);
            const double zi = B.dinv[i] * ri;
            B.r[i] = ri;
            B.z[i] = zi;
            acc[0] = fma(ri, zi, acc[0]);
            acc[1] = fma(ri, ri, acc[1]);
        });
        block_sum<2>(acc, red);
        if (threadIdx.x == 0) {
            B.part[4 * kMaxGrid + blockIdx.x] = acc[0];
            B.part[5 * kMaxGrid + blockIdx.x] = acc[1];
        }
        if (!grid_sync(ctrl, gridDim.x)) return;
        const double rz_new = grid_reduce(B.part, 4, gridDim.x, red + 96);
        rr = grid_reduce(B.part, 5, gridDim.x, red + 96);
        ++it;
        if (rr <= stop) {
            // confirm with the true residual
            double bb2;
            if (!setup_phase(op, B, red, bb2, rz, rr, ctrl)) return;
            if (rr <= stop) { result = 1; break; }
            if (++restarts > max_restarts) { result = 0; break; }
            first = true;
            beta = 0.0;
            if (it >= maxit) { result = 0; break; }
            continue;
        }
        if (it >= maxit) { result = 0; break; }
        beta = rz_new / rz;
        rz = rz_new;
        first = false;
    }
    if (result == 0 && it >= maxit) {
        // report the true residual of the last iterate
        double bb2, rz2, rr2;
        if (!setup_phase(op, B, red, bb2, rz2, rr2, ctrl)) return;
        rr = rr2;
    }
    if (lead) {
        ctrl->iters = it;
        ctrl->restarts = restarts;
        ctrl->converged = result;
        ctrl->early = 0;
        ctrl->relres = sqrt(rr / bb);
        if (result == -1) atomicCAS(&ctrl->status, LC_OK, LC_ERR_BREAKDOWN);
    }
}

__global__ void csr_dinv_kernel(Csr c, double *dinv) {
    const int32_t n = c.n_dev ? *c.n_dev : c.n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        const int32_t e1 = c.rp[i + 1];
        for (int32_t e = c.rp[i]; e < e1; ++e)
            if (c.ci[e] == i) d = c.av[e];
        dinv[i] = 1.0 / d;
    }
}

__global__ void reset_ctrl_kernel(Ctrl *ctrl) {
    ctrl->bar_count = 0;
    ctrl->iters = 0;
    ctrl->restarts = 0;
    ctrl->converged = 0;
    ctrl->early = 0;
}

__global__ void dinv_stencil_kernel(int64_t n, const double *D, double *dinv, float *D32, const double *Tx,
                                    const double *Ty, const double *Tz, float *Tx32, float *Ty32, float *Tz32,
                                    float *dinv32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = D[i];
        dinv[i] = 1.0 / d;
        if (D32) {
            D32[i] = (float)d;
            Tx32[i] = (float)Tx[i];
            Ty32[i] = (float)Ty[i];
            if (Tz) Tz32[i] = (float)Tz[i];
            dinv32[i] = 1.0f / (float)d;
        }
    }
}

// Validation: D > 0 everywhere and every interior face conductance > 0.
__global__ void check_stencil_kernel(Stencil s, int *bad) {
    const int64_t sxy = (int64_t)s.nx * s.ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % s.nx), yy = (int)((i / s.nx) % s.ny), zz = (int)(i / sxy);
        bool ok = s.D[i] > 0.0;
        if (xx + 1 < s.nx) ok = ok && s.Tx[i] > 0.0;
        if (yy + 1 < s.ny) ok = ok && s.Ty[i] > 0.0;
        if (s.dim == 3 && zz + 1 < s.nz) ok = ok && s.Tz[i] > 0.0;
        if (!ok) atomicExch(bad, 1);
    }
}

// Validation: rowptr monotone and in range, columns in range and strictly
// ascending within each row, diagonal present and positive.
__global__ void check_csr_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *av, int *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e0 = rp[i], e1 = rp[i + 1];
        bool ok = e0 >= 0 && e1 >= e0 && e1 <= rp[n];
        bool diag = false;
        int32_t prev = -1;
        for (int32_t e = e0; ok && e < e1; ++e) {
            const int32_t j = ci[e];
            if (j < 0 || j >= n || j <= prev) ok = false;
            prev = j;
            if (j == i) diag = av[e] > 0.0;
        }
        if (!ok || !diag) atomicExch(bad, 1);
    }
}

template <class OP>
int pcg_grid(const void *kernel, int64_t units, int cap) {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kPcgThreads, 0);
    int64_t g = (int64_t)sms * (per < 1 ? 1 : per);
    if (cap > 0 && g > cap) g = cap;
    if (g > units) g = units;
    if (g > kMaxGrid) g = kMaxGrid;
    return (int)(g < 1 ? 1 : g);
}

// minblocks = the register budget asked of the compiler (blocks of 256
// threads that must fit on one SM): 1 = unconstrained, 2..4 = at most
// 128 / 85 / 64 registers per thread.
template <class OP>
const void *pcg_kernel_for(int minblocks) {
    switch (minblocks) {
        case 2: return (const void *)pcg_kernel<OP, 2>;
        case 3: return (const void *)pcg_kernel<OP, 3>;
        case 4: return (const void *)pcg_kernel<OP, 4>;
        default: return (const void *)pcg_kernel<OP, 1>;
    }
}

template <class OP>
cudaError_t launch_coop(const OP &op, int64_t units, const Bufs &B, double tol, int maxit, int max_restarts,
                        Ctrl *ctrl, int cap, int minblocks, cudaStream_t s) {
    const void *k = pcg_kernel_for<OP>(minblocks);
    const int grid = pcg_grid<OP>(k, units, cap);
    reset_ctrl_kernel<<<1, 1, 0, s>>>(ctrl);
    note_launches(1);
    OP o = op;
    Bufs b = B;
    double t = tol;
    int mi = maxit, mr = max_restarts;
    Ctrl *c = ctrl;
    void *args[] = {&o, &b, &t, &mi, &mr, &c};
    note_launches(1);
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kPcgThreads), args, 0, s);
}

}  // namespace

cudaError_t launch_pcg_stencil(const Stencil &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                               cudaStream_t s) {
    Bufs B;
    B.b = a.b; B.x = a.x; B.r = w.r; B.z = w.z; B.q = w.q; B.p0 = w.p0; B.p1 = w.p1;
    B.dinv = op.dinv; B.part = w.partials;
    if (op.dim == 3) {
        Op3D o{op};
        const int64_t units = (int64_t)((op.nx + kTileX - 1) / kTileX) * ((op.ny + kTileY - 1) / kTileY) *
                              ((op.nz + kTileZ - 1) / kTileZ);
        return launch_coop(o, units, B, a.tol, a.maxit, a.max_restarts, ctrl, grid_hint, 1, s);
    }
    // two cells per lane (16-byte vectors) when every row starts 16-byte aligned
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    const bool vec = op.nx % 2 == 0 && al16(op.D) && al16(op.Tx) && al16(op.Ty);
    const int warps_per_block = kPcgThreads / 32;
    if (vec) {
        Op2DW<2> o{op};
        // at least 4 rows per warp so the recomputed halo rows stay a small overhead
        const int64_t units = ((int64_t)((op.nx + 63) / 64) * op.ny + 4 * warps_per_block - 1) / (4 * warps_per_block);
        return launch_coop(o, units, B, a.tol, a.maxit, a.max_restarts, ctrl, grid_hint, a.minblocks, s);
    }
    Op2DW<1> o{op};
    const int64_t units = ((int64_t)((op.nx + 31) / 32) * op.ny + 4 * warps_per_block - 1) / (4 * warps_per_block);
    return launch_coop(o, units, B, a.tol, a.maxit, a.max_restarts, ctrl, grid_hint, a.minblocks, s);
}

cudaError_t launch_pcg_csr(const Csr &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint, cudaStream_t s) {
    // the row count may live on the device (extracted subsystem): the kernel
    // is sized for the capacity op.n and reads the actual count itself
    csr_dinv_kernel<<<152 * 4, 256, 0, s>>>(op, w.dinv);
    note_launches(1);
    Bufs B;
    B.b = a.b; B.x = a.x; B.r = w.r; B.z = w.z; B.q = w.q; B.p0 = w.p0; B.p1 = w.p1;
    B.dinv = w.dinv; B.part = w.partials;
    OpCsr o{op, op.n};
    const int64_t units = (op.n + kPcgThreads - 1) / kPcgThreads;
    return launch_coop(o, units, B, a.tol, a.maxit, a.max_restarts, ctrl, grid_hint, 1, s);
}

cudaError_t launch_dinv_stencil(int64_t n, const double *D, double *dinv, float *D32, const double *Tx,
                                const double *Ty, const double *Tz, float *Tx32, float *Ty32, float *Tz32,
                                float *dinv32, cudaStream_t s) {
    dinv_stencil_kernel<<<152 * 8, 256, 0, s>>>(n, D, dinv, D32, Tx, Ty, Tz, Tx32, Ty32, Tz32, dinv32);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_check_stencil(const Stencil &op, int *bad, cudaStream_t s) {
    check_stencil_kernel<<<152 * 8, 256, 0, s>>>(op, bad);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_check_csr(int32_t n, const int32_t *rp, const int32_t *ci, const double *av, int *bad,
                             cudaStream_t s) {
    check_csr_kernel<<<152 * 8, 256, 0, s>>>(n, rp, ci, av, bad);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace lc
