// lc_pcg_impl.cuh -- the persistent Krylov kernels shared by the solver
// translation units (lc_pcg.cu: 2D FP64 and set-up; lc_pcg_mixed.cu: 2D
// mixed precision; lc_pcg3d.cu: 3D; lc_pcgcsr.cu: CSR), which each
// instantiate the operators they launch.  Everything here has internal
// linkage.
//
// Jacobi-preconditioned conjugate gradients as ONE persistent cooperative
// kernel per solve (the Krylov solver of Alg 1, steps 5 and 11), in FP64,
// and FP32 inner solves inside FP64 iterative refinement.
//
// Per CG iteration two grid-wide phases, each closed by a bounded grid
// barrier and a deterministic fixed-slot reduction (every block sums the
// same block partials in the same order, so every block takes the same
// decisions):
//
//   phase A  p = z + beta p_old          (computed where it is needed, halos
//            q = A p, partial p.q          included, so no extra barrier)
//            store p (ping-pong buffer) and q
//   phase B  alpha = rz / pq; x += alpha p; r -= alpha q; z = dinv r;
//            partials r.z and r.r
//
// z is stored so that phase A reads one vector where it would read r and
// dinv.  FP64 solve: the stopping test ||r||^2 <= tol^2 ||b||^2 is taken on
// the recurrence residual, confirmed with the true residual b - A x, and the
// iteration restarts from the true residual when that misses (at most
// max_restarts).  The test on the starting iterate happens in the set-up
// phase: a converged start (Alg 1 step 8, the local solution x~ already good
// enough) costs one residual pass and no iteration.
//
// Mixed precision (iterative refinement): r = b - A x in FP64; stop if
// ||r|| <= tol ||b||; else solve fl32(A) d = fl32(r/||r||) by FP32 Jacobi-PCG
// from d = 0 until its residual fell by inner_tol (vectors and per-thread
// sums in FP32, only the cross-block sums in FP64); x += ||r|| d in FP64;
// repeat.  All of it in one launch.
//
// FP64 stencil solves (by default) iterate on the symmetrically scaled
// system S A S x^ = S b, S = D^-1/2, x = S x^: its diagonal is 1, so the
// Jacobi preconditioner is the identity, z = r^, and no D or dinv is read in
// the loop -- the same preconditioned iteration in exact arithmetic (the
// Jacobi-PCG iterates x_k are S times the scaled iterates).  Its stopping
// norm ||r||^2 = sum D r^^2 is summed in FP32 from the bits of r^ (no FP64
// instruction) and confirmed in FP64 by the true-residual pass like every
// other convergence.  The default 2D and 3D variants also take p.q and the
// block sums on FP32 pairs (split_f2, grid_sums_pair) and carry the update
// x += alpha p into the next iteration's phase A, which loads p anyway.
//
// Data movement per cell and CG iteration, 2D: phase A reads z, p_old, D,
// Tx, Ty and writes p, q; phase B reads x, p, r, q, dinv and writes x, r, z:
// 120 B in FP64, 60 B in FP32 (3D: 128 B / 64 B).  The default scaled 2D
// FP64 kernel: phase A reads r^, p_old, x^, Tx^, Ty^ and writes p, q, x^;
// phase B reads r^, q, fl32(D) and writes r^: 92 B, 8 FP64 instructions.
#pragma once

#include "lc_internal.cuh"

namespace lc {

namespace {

constexpr int kPcgThreads = 256;
constexpr int kTileX = 32, kTileY = 8, kTileZ = 16;   // 3D unit

// N consecutive values of type T moved as one vector access (N = 1, 2, 4;
// 4 only for float): 16-byte accesses for double2 / float4.
template <typename T, int N> struct VecType { using type = T; };
template <> struct VecType<double, 2> { using type = double2; };
template <> struct VecType<float, 2> { using type = float2; };
template <> struct VecType<float, 4> { using type = float4; };

template <typename T, int N>
union VecU {
    typename VecType<T, N>::type v;
    T e[N];
};

// four doubles move as two double2 accesses
template <typename T, int N>
__device__ __forceinline__ void vld(const T *a, T (&out)[N]) {
    if constexpr (N == 4 && sizeof(T) == 8) {
        const double2 lo = reinterpret_cast<const double2 *>(a)[0], hi = reinterpret_cast<const double2 *>(a)[1];
        out[0] = lo.x; out[1] = lo.y; out[2] = hi.x; out[3] = hi.y;
    } else {
        VecU<T, N> u;
        u.v = *reinterpret_cast<const typename VecType<T, N>::type *>(a);
#pragma unroll
        for (int k = 0; k < N; ++k) out[k] = u.e[k];
    }
}
template <typename T, int N>
__device__ __forceinline__ void vld_cg(const T *a, T (&out)[N]) {
    if constexpr (N == 4 && sizeof(T) == 8) {
        const double2 lo = __ldcg(reinterpret_cast<const double2 *>(a)), hi = __ldcg(reinterpret_cast<const double2 *>(a) + 1);
        out[0] = lo.x; out[1] = lo.y; out[2] = hi.x; out[3] = hi.y;
    } else {
        VecU<T, N> u;
        u.v = __ldcg(reinterpret_cast<const typename VecType<T, N>::type *>(a));
#pragma unroll
        for (int k = 0; k < N; ++k) out[k] = u.e[k];
    }
}
template <typename T, int N>
__device__ __forceinline__ void vst(T *a, const T (&in)[N]) {
    if constexpr (N == 4 && sizeof(T) == 8) {
        reinterpret_cast<double2 *>(a)[0] = make_double2(in[0], in[1]);
        reinterpret_cast<double2 *>(a)[1] = make_double2(in[2], in[3]);
    } else {
        VecU<T, N> u;
#pragma unroll
        for (int k = 0; k < N; ++k) u.e[k] = in[k];
        *reinterpret_cast<typename VecType<T, N>::type *>(a) = u.v;
    }
}

template <typename T>
struct Vecs {
    const T *b;
    T *x, *r, *z, *q, *p0, *p1;
    const T *dinv;
    T *xu;   // scaled solves: the caller's x (x holds x^ = D^1/2 x in a workspace)
};

// A float within 2^-23 (relative) of |v| * 2^-nscale, built from the bits of
// v with integer instructions only (no FP64 instruction): enough for a
// stopping norm, which is confirmed in FP64 afterwards.  nscale moves the
// values the norm sums into FP32's range; below that range it gives 0, above
// it (or for NaN) +inf.
__device__ __forceinline__ float approx_abs_f32(double v, int nscale) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023 + 127 - nscale;
    if (e <= 0) return 0.0f;
    if (e >= 255) return __int_as_float(0x7f800000);
    return __uint_as_float(((unsigned)e << 23) | (unsigned)((bits >> 29) & 0x7fffff));
}

// Dot products on FP32 pairs.  GB300 issues FP64 at 1/64 of its FP32 rate and
// the FP64 pipe is what bounds the scaled 2D iteration, while most issue
// slots sit idle; so its dot products can run on the FP32 and integer pipes:
// v * 2^-ns is split into hi + lo (the top 24 and the next 23 significand
// bits, 47 of v's 53) from v's bits, products and sums use the error-free
// FP32 transformations (Dekker's product through FMA, Knuth's two-sum), and
// the pair accumulates with a relative error near 2^-45 per term -- far
// below what alpha and beta need (the iterates then differ from FP64 sums in
// rounding only).  hi is the approx_abs_f32 value with v's sign.  Values
// below 2^-126 (scaled) give 0, above FP32's range +-inf.
__device__ __forceinline__ void split_f2(double v, int ns, float &hi, float &lo) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const unsigned sign = (unsigned)(bits >> 32) & 0x80000000u;
    const int e = (int)((bits >> 52) & 0x7ff) - 1023 - ns;   // unbiased exponent of v 2^-ns
    const unsigned mh = (unsigned)(bits >> 29) & 0x7fffffu, ml = (unsigned)(bits >> 6) & 0x7fffffu;
    hi = e + 127 <= 0 ? 0.0f
                      : __uint_as_float(sign | (e + 127 >= 255 ? 0x7f800000u : ((unsigned)(e + 127) << 23) | mh));
    // ml 2^(e-46) = (1.ml - 1) 2^(e-23), the power of two (with v's sign) from bits
    lo = e + 104 <= 0 || e + 127 >= 255
             ? 0.0f
             : __fmul_rn(__fsub_rn(__uint_as_float(0x3f800000u | ml), 1.0f),
                         __uint_as_float(sign | ((unsigned)(e + 104) << 23)));
}
// (sh, sl) += (ah + al)(bh + bl), dropping al bl
__device__ __forceinline__ void f2_add_prod(float ah, float al, float bh, float bl, float &sh, float &sl) {
    const float p = __fmul_rn(ah, bh);
    const float t = fmaf(al, bh, fmaf(ah, bl, fmaf(ah, bh, -p)));   // the product's error and cross terms
    const float s = __fadd_rn(sh, p);
    const float bv = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, t));
}
// the pair's value times 2^(2 ns), in FP64 (once per thread and phase)
__device__ __forceinline__ double f2_value(float sh, float sl, int ns) {
    return ldexp((double)sh + (double)sl, 2 * ns);
}

template <typename T>
struct Coef {
    const T *D, *Tx, *Ty, *Tz;
};

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// Phase B of a Jacobi-PCG iteration over the operator's cells:
// x += alpha p, r -= alpha q, z = dinv r; sums r.z and r.r.
template <class OP, typename T>
__device__ __forceinline__ void phaseB_generic(const OP &op, const Vecs<T> &V, const T *p, T alpha, T (&acc)[2]) {
    op.each_cell([&](int64_t i) {
        // every load before the first store (which the compiler cannot prove
        // apart from them)
        const T pi = p[i], qi = V.q[i], xi = V.x[i], r0 = V.r[i], di = V.dinv[i];
        V.x[i] = fmaT(alpha, pi, xi);
        const T ri = fmaT(-alpha, qi, r0);
        const T zi = di * ri;
        V.r[i] = ri;
        V.z[i] = zi;
        acc[0] = fmaT(ri, zi, acc[0]);
        acc[1] = fmaT(ri, ri, acc[1]);
    });
}

// -------------------------------------------------------------- operators
//
// Every operator provides, for the calling block:
//   setup_block     r = b - A x (and z = dinv r if z is given) over its cells;
//                   sums b.b, r.z, r.r
//   phaseA_block    p = z + beta p_old, q = A p over its cells; sums p.q
//   each_cell(f)    f(i) for its cells, in the same cell-to-thread mapping as
//                   phase A, so the p and q a thread stored are the ones it
//                   reads back.

// 2D, warp-independent: the grid is cut into column strips of 32*CPL cells,
// one lane owning CPL adjacent columns (CPL = 2 when rows start aligned, so
// loads/stores are pairs; 4 in the scaled FP64 solve when nx is a multiple
// of 4).  The strip-major list of (strip, row) items is split evenly over
// all warps of the grid and every warp marches down its own rows: p of the
// rows above and below in registers, x-neighbours through warp shuffles, the
// one-cell halo at either end of the strip recomputed by lanes 0 and 31.  No
// block barrier, no shared memory.
//
// UNIT = the symmetrically scaled system S A S x^ = S b, S = D^-1/2, x = S x^
// (Jacobi-PCG on A in exact arithmetic): unit diagonal, z = r^ (no multiply,
// no separate vector), r.z = r^.r^; the stopping norm ||r||^2 = sum D r^^2
// is accumulated in FP32 from approx_abs_f32 and confirmed in FP64 by the
// true-residual pass.  c holds D (for that pass) and the scaled faces.
// F2D: p.q and the block sums on FP32 pairs.  DX: x += alpha p applied in
// the next iteration's phase A (on the p_old it loads) and by flush_x after
// the last one.
template <typename T, int CPL, bool UNIT = false, bool F2D = false, bool DX = false>
struct Op2DW {
    Stencil s;
    Coef<T> c;
    const double *sc = nullptr, *sq = nullptr;   // UNIT: D^-1/2, D^1/2
    const float *d32 = nullptr;                  // UNIT, FP64: fl32(D 2^-2h); FP32: fl32(D^1/2) (stopping norm)
    const int *dexp = nullptr;                   // UNIT: h = (*dexp - 1023) >> 1
    static constexpr int kSW = 32 * CPL;
    static constexpr int kSmem = 1;
    static constexpr bool kAnyBlock = true;   // strips are per warp: any block size
    static constexpr bool kScaled = UNIT;
    static constexpr bool kPairDots = F2D;    // phase A's block sums on FP32 pairs
    static constexpr bool kDeferX = DX;       // x += alpha p rides on the next phase A
    static_assert(!DX || UNIT, "the deferred x update is built for the scaled system");
    static_assert(!F2D || (UNIT && sizeof(T) == 8), "pair dot products are built for the scaled FP64 solve");
    __device__ bool skipped() const { return false; }
    __device__ void resolve() {}
    __device__ int dn_shift() const { return UNIT ? (*dexp - 1023) >> 1 : 0; }
    __device__ void prologue(const Vecs<T> &V) const {
        if (UNIT) each_cell([&](int64_t i) { V.x[i] = V.xu[i] * sq[i]; });
    }
    __device__ void epilogue(const Vecs<T> &V) const {
        if (UNIT) each_cell([&](int64_t i) { V.xu[i] = V.x[i] * sc[i]; });
    }
    __device__ void zero_solution(const Vecs<T> &V) const {
        each_cell([&](int64_t i) { (UNIT ? V.xu : V.x)[i] = T(0); });
    }
    // rows of CPL-wide vector loads and stores (nx is a multiple of CPL)
    __device__ void phaseB_block(const Vecs<T> &V, const T *p, T alpha, T (&acc)[2], int nscale) const {
        const int lane = threadIdx.x & 31;
        float rrf = 0.f;
        each_segment([&](int x0, int y0, int y1) {
            const int xa = x0 + CPL * lane;
            if (xa >= s.nx) return;
#pragma unroll 2
            for (int y = y0; y < y1; ++y) {
                const int64_t i = (int64_t)y * s.nx + xa;
                T pv[CPL], qv[CPL], xv[CPL], rv[CPL];
                if constexpr (!DX) {
                    vld<T, CPL>(p + i, pv);
                    vld<T, CPL>(V.x + i, xv);
                }
                vld<T, CPL>(V.q + i, qv);
                vld<T, CPL>(V.r + i, rv);
                if (UNIT) {
                    float dv[CPL];
                    vld<float, CPL>(d32 + i, dv);
#pragma unroll
                    for (int k = 0; k < CPL; ++k) {
                        if constexpr (!DX) xv[k] = fmaT(alpha, pv[k], xv[k]);
                        rv[k] = fmaT(-alpha, qv[k], rv[k]);
                        acc[0] = fmaT(rv[k], rv[k], acc[0]);
                        if constexpr (sizeof(T) == 8) {   // FP64: sum D r^^2 from the bits of r^
                            const float f = approx_abs_f32((double)rv[k], nscale);
                            rrf = fmaf(dv[k] * f, f, rrf);
                        } else {                          // FP32: sum (D^1/2 r^)^2 directly
                            const float t = dv[k] * rv[k];
                            rrf = fmaf(t, t, rrf);
                        }
                    }
                } else {
                    T dv[CPL], zv[CPL];
                    vld<T, CPL>(V.dinv + i, dv);
#pragma unroll
                    for (int k = 0; k < CPL; ++k) {
                        xv[k] = fmaT(alpha, pv[k], xv[k]);
                        rv[k] = fmaT(-alpha, qv[k], rv[k]);
                        zv[k] = dv[k] * rv[k];
                        acc[0] = fmaT(rv[k], zv[k], acc[0]);
                        acc[1] = fmaT(rv[k], rv[k], acc[1]);
                    }
                    vst<T, CPL>(V.z + i, zv);
                }
                if constexpr (!DX) vst<T, CPL>(V.x + i, xv);
                vst<T, CPL>(V.r + i, rv);
            }
        });
        if (UNIT) acc[1] = (T)rrf;
    }
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
    template <class F>
    __device__ __forceinline__ void each_cell(F f) const {
        const int lane = threadIdx.x & 31;
        each_segment([&](int x0, int y0, int y1) {
            const int xa = x0 + CPL * lane;
#pragma unroll 2
            for (int y = y0; y < y1; ++y)
#pragma unroll
                for (int k = 0; k < CPL; ++k)
                    if (xa + k < s.nx) f((int64_t)y * s.nx + xa + k);
        });
    }
    __device__ void setup_block(const Vecs<T> &V, T &bb, T &rz, T &rr) const {
        each_cell([&](int64_t i) {
            const int xx = (int)(i % s.nx), y = (int)(i / s.nx);
            T ax = UNIT ? ldcg(V.x + i) : c.D[i] * ldcg(V.x + i);
            if (y > 0) ax = fmaT(-c.Ty[i - s.nx], ldcg(V.x + i - s.nx), ax);
            if (xx > 0) ax = fmaT(-c.Tx[i - 1], ldcg(V.x + i - 1), ax);
            if (xx + 1 < s.nx) ax = fmaT(-c.Tx[i], ldcg(V.x + i + 1), ax);
            if (y + 1 < s.ny) ax = fmaT(-c.Ty[i], ldcg(V.x + i + s.nx), ax);
            const T bi = V.b[i];
            bb = fmaT(bi, bi, bb);
            if (UNIT) {   // r^ = S b - A^ x^;  ||r||^2 = sum D r^^2
                const T ri = (T)sc[i] * bi - ax;
                V.r[i] = ri;
                rz = fmaT(ri, ri, rz);
                rr = fmaT(c.D[i] * ri, ri, rr);
                return;
            }
            const T ri = bi - ax;
            V.r[i] = ri;
            rr = fmaT(ri, ri, rr);
            if (V.z) {
                const T zi = V.dinv[i] * ri;
                V.z[i] = zi;
                rz = fmaT(ri, zi, rz);
            }
        });
    }
    __device__ __forceinline__ T pnew1(const Vecs<T> &V, const T *pold, bool first, T beta, int64_t i) const {
        const T zi = ldcg(V.z + i);
        return first ? zi : fmaT(beta, ldcg(pold + i), zi);
    }
    // p = z + beta p_old; DX and own: also x += ax p_old (the last
    // iteration's update, on the p_old this load brings anyway)
    __device__ __forceinline__ void pnew(const Vecs<T> &V, const T *pold, bool first, T beta, int64_t i,
                                        T (&p)[CPL], T ax = T(0), bool own = false) const {
        vld_cg<T, CPL>(V.z + i, p);
        if (!first) {
            T o[CPL];
            vld_cg<T, CPL>(pold + i, o);
            if constexpr (DX) {
                if (own) {
                    T xv[CPL];
                    vld<T, CPL>(V.x + i, xv);
#pragma unroll
                    for (int k = 0; k < CPL; ++k) xv[k] = fmaT(ax, o[k], xv[k]);
                    vst<T, CPL>(V.x + i, xv);
                }
            }
#pragma unroll
            for (int k = 0; k < CPL; ++k) p[k] = fmaT(beta, o[k], p[k]);
        }
    }
    // DX: the update of x the last phase A would have carried
    __device__ void flush_x(const Vecs<T> &V, const T *p, T alpha) const {
        const int lane = threadIdx.x & 31;
        each_segment([&](int x0, int y0, int y1) {
            const int xa = x0 + CPL * lane;
            if (xa >= s.nx) return;
            for (int y = y0; y < y1; ++y) {
                const int64_t i = (int64_t)y * s.nx + xa;
                T pv[CPL], xv[CPL];
                vld<T, CPL>(p + i, pv);
                vld<T, CPL>(V.x + i, xv);
#pragma unroll
                for (int k = 0; k < CPL; ++k) xv[k] = fmaT(alpha, pv[k], xv[k]);
                vst<T, CPL>(V.x + i, xv);
            }
        });
    }
    __device__ __forceinline__ void load(const T *a, int64_t i, T (&v)[CPL]) const { vld<T, CPL>(a + i, v); }
    // F2D: p.q as an FP32 pair of the values scaled by 2^-nscale (a sum
    // scaled by 2^-2 nscale), into pair[0..2) if given, else added to pq
    __device__ void phaseA_block(const Vecs<T> &V, const T *pold, T *pout, bool first, T beta, T &pq, T *,
                                 int nscale, float *pair = nullptr, T ax = T(0)) const {
        const int lane = threadIdx.x & 31;
        float fh = 0.f, fl = 0.f;
        each_segment([&](int x0, int y0, int y1) {
            const int xa = x0 + CPL * lane;          // first column of this lane
            const bool act = xa < s.nx;               // nx is a multiple of CPL: all CPL cells valid
            const int hx = lane == 0 ? x0 - 1 : x0 + kSW;
            const bool hact = (lane == 0 && x0 > 0) || (lane == 31 && x0 + kSW < s.nx);
            T pm[CPL], pc[CPL], pn[CPL], tym[CPL];
#pragma unroll
            for (int k = 0; k < CPL; ++k) { pm[k] = T(0); pc[k] = T(0); tym[k] = T(0); }
            if (act) {
                const int64_t i0 = (int64_t)y0 * s.nx + xa;
                pnew(V, pold, first, beta, i0, pc, ax, true);
                if (y0 > 0) {
                    pnew(V, pold, first, beta, i0 - s.nx, pm);
                    load(c.Ty, i0 - s.nx, tym);
                }
            }
            for (int y = y0; y < y1; ++y) {
                const int64_t i = (int64_t)y * s.nx + xa;
                T d[CPL], tx[CPL], typ[CPL];
                T txw0 = T(0), ph = T(0);
#pragma unroll
                for (int k = 0; k < CPL; ++k) { pn[k] = T(0); d[k] = T(0); tx[k] = T(0); typ[k] = T(0); }
                if (act) {
                    if (y + 1 < s.ny) {
                        pnew(V, pold, first, beta, i + s.nx, pn, ax, y + 1 < y1);
                        load(c.Ty, i, typ);
                    }
                    if (!UNIT) load(c.D, i, d);
                    load(c.Tx, i, tx);
                    if (lane == 0 && x0 > 0) txw0 = c.Tx[i - 1];
                }
                if (hact) ph = pnew1(V, pold, first, beta, (int64_t)y * s.nx + hx);
                const T tx_last_up = __shfl_up_sync(kFull, tx[CPL - 1], 1);
                const T pc_last_up = __shfl_up_sync(kFull, pc[CPL - 1], 1);
                const T pc_first_dn = __shfl_down_sync(kFull, pc[0], 1);
                if (!act) continue;
                T txw[CPL], txe[CPL], pw[CPL], pe[CPL];
                txw[0] = lane == 0 ? txw0 : tx_last_up;
                pw[0] = lane == 0 ? ph : pc_last_up;
#pragma unroll
                for (int k = 1; k < CPL; ++k) { txw[k] = tx[k - 1]; pw[k] = pc[k - 1]; }
#pragma unroll
                for (int k = 0; k < CPL - 1; ++k) { txe[k] = tx[k]; pe[k] = pc[k + 1]; }
                const bool last_col = xa + CPL >= s.nx;
                txe[CPL - 1] = last_col ? T(0) : tx[CPL - 1];
                pe[CPL - 1] = lane == 31 ? ph : pc_first_dn;
                T q[CPL];
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    T qi = UNIT ? pc[k] : d[k] * pc[k];
                    qi = fmaT(-tym[k], pm[k], qi);
                    qi = fmaT(-txw[k], pw[k], qi);
                    qi = fmaT(-txe[k], pe[k], qi);
                    qi = fmaT(-typ[k], pn[k], qi);
                    q[k] = qi;
                    if constexpr (F2D) {
                        float ph_, pl_, qh_, ql_;
                        split_f2((double)pc[k], nscale, ph_, pl_);
                        split_f2((double)qi, nscale, qh_, ql_);
                        f2_add_prod(ph_, pl_, qh_, ql_, fh, fl);
                    } else {
                        pq = fmaT(pc[k], qi, pq);
                    }
                }
                vst<T, CPL>(pout + i, pc);
                vst<T, CPL>(V.q + i, q);
#pragma unroll
                for (int k = 0; k < CPL; ++k) { tym[k] = typ[k]; pm[k] = pc[k]; pc[k] = pn[k]; }
            }
        });
        if constexpr (F2D) {
            if (pair) { pair[0] = fh; pair[1] = fl; }
            else pq += f2_value(fh, fl, nscale);
        }
    }
};

// 3D: units of kTileX x kTileY columns marching kTileZ planes; p of each
// plane (tile + one-cell xy halo) built once into shared memory (four
// rotating planes: one barrier per plane), z-neighbours from the planes
// above and below.
//
// UNIT = the symmetrically scaled system, as for Op2DW: unit diagonal, z = r^,
// stopping norm sum D r^^2 in FP32, c holding D (residual passes) and the
// scaled faces.
template <typename T, bool UNIT = false, bool F2D = false, bool DX = false>
struct Op3D {
    Stencil s;
    Coef<T> c;
    const double *sc = nullptr, *sq = nullptr;   // UNIT: D^-1/2, D^1/2
    const float *d32 = nullptr;                  // UNIT, FP64: fl32(D 2^-2h); FP32: fl32(D^1/2)
    const int *dexp = nullptr;                   // UNIT, FP64: h = (*dexp - 1023) >> 1
    static constexpr int kSmem = 2 * (kTileX + 2) * (kTileY + 2);
    static constexpr bool kAnyBlock = false;   // one tile per block of kPcgThreads
    static constexpr bool kScaled = UNIT;
    static constexpr bool kPairDots = F2D;     // p.q and the block sums on FP32 pairs (as Op2DW)
    static constexpr bool kDeferX = DX;        // x += alpha p rides on the next phase A (as Op2DW)
    static_assert(!DX || UNIT, "the deferred x update is built for the scaled system");
    static_assert(!F2D || (UNIT && sizeof(T) == 8), "pair dot products are built for the scaled FP64 solve");
    __device__ bool skipped() const { return false; }
    __device__ void resolve() {}
    __device__ int dn_shift() const { return UNIT ? (*dexp - 1023) >> 1 : 0; }
    __device__ void prologue(const Vecs<T> &V) const {
        if (UNIT) each_cell([&](int64_t i) { V.x[i] = V.xu[i] * sq[i]; });
    }
    __device__ void epilogue(const Vecs<T> &V) const {
        if (UNIT) each_cell([&](int64_t i) { V.xu[i] = V.x[i] * sc[i]; });
    }
    __device__ void zero_solution(const Vecs<T> &V) const {
        each_cell([&](int64_t i) { (UNIT ? V.xu : V.x)[i] = T(0); });
    }
    // Phase B over the own column of every unit, kBz planes at a time with
    // all their loads issued before the first store (the compiler keeps a
    // store through one vector pointer ahead of a later load through
    // another, so a plane-by-plane loop would wait for every plane's loads
    // in turn); the per-thread sums keep the plane order.
    static constexpr int kBz = 4;
    __device__ void phaseB_block(const Vecs<T> &V, const T *p, T alpha, T (&acc)[2], int nscale) const {
        float rrf = 0.f;
        const int64_t nu = units();
        const int64_t sxy = (int64_t)s.nx * s.ny;
        for (int64_t u = blockIdx.x; u < nu; u += gridDim.x) {
            int x0, y0, z0;
            origin(u, x0, y0, z0);
            const int xx = x0 + (threadIdx.x % kTileX), yy = y0 + (threadIdx.x / kTileX);
            if (xx >= s.nx || yy >= s.ny) continue;
            const int z1 = min(z0 + kTileZ, s.nz);
            const int64_t col = xx + (int64_t)s.nx * yy;
            for (int zb = z0; zb < z1; zb += kBz) {
                T qv[kBz], rv[kBz], pv[kBz], xv[kBz], dv[kBz];
                float fv[kBz];
#pragma unroll
                for (int k = 0; k < kBz; ++k) {
                    if (zb + k >= z1) break;
                    const int64_t i = col + sxy * (zb + k);
                    qv[k] = V.q[i];
                    rv[k] = V.r[i];
                    if (UNIT) fv[k] = d32[i];
                    else dv[k] = V.dinv[i];
                    if (!UNIT || !DX) { pv[k] = p[i]; xv[k] = V.x[i]; }
                }
#pragma unroll
                for (int k = 0; k < kBz; ++k) {
                    if (zb + k >= z1) break;
                    const int64_t i = col + sxy * (zb + k);
                    if (!UNIT || !DX) V.x[i] = fmaT(alpha, pv[k], xv[k]);
                    const T ri = fmaT(-alpha, qv[k], rv[k]);
                    V.r[i] = ri;
                    if constexpr (!UNIT) {
                        const T zi = dv[k] * ri;
                        V.z[i] = zi;
                        acc[0] = fmaT(ri, zi, acc[0]);
                        acc[1] = fmaT(ri, ri, acc[1]);
                    } else {
                        acc[0] = fmaT(ri, ri, acc[0]);
                        if constexpr (sizeof(T) == 8) {
                            const float f = approx_abs_f32((double)ri, nscale);
                            rrf = fmaf(fv[k] * f, f, rrf);
                        } else {
                            const float t = fv[k] * ri;
                            rrf = fmaf(t, t, rrf);
                        }
                    }
                }
            }
        }
        if constexpr (UNIT) acc[1] = (T)rrf;
    }
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
    __device__ void setup_block(const Vecs<T> &V, T &bb, T &rz, T &rr) const {
        const int64_t sxy = (int64_t)s.nx * s.ny;
        each_cell([&](int64_t i) {
            const int xx = (int)(i % s.nx), yy = (int)((i / s.nx) % s.ny), zz = (int)(i / sxy);
            T ax = UNIT ? ldcg(V.x + i) : c.D[i] * ldcg(V.x + i);
            if (zz > 0) ax = fmaT(-c.Tz[i - sxy], ldcg(V.x + i - sxy), ax);
            if (yy > 0) ax = fmaT(-c.Ty[i - s.nx], ldcg(V.x + i - s.nx), ax);
            if (xx > 0) ax = fmaT(-c.Tx[i - 1], ldcg(V.x + i - 1), ax);
            if (xx + 1 < s.nx) ax = fmaT(-c.Tx[i], ldcg(V.x + i + 1), ax);
            if (yy + 1 < s.ny) ax = fmaT(-c.Ty[i], ldcg(V.x + i + s.nx), ax);
            if (zz + 1 < s.nz) ax = fmaT(-c.Tz[i], ldcg(V.x + i + sxy), ax);
            const T bi = V.b[i];
            bb = fmaT(bi, bi, bb);
            if (UNIT) {   // r^ = S b - A^ x^;  ||r||^2 = sum D r^^2
                const T rh = (T)sc[i] * bi - ax;
                V.r[i] = rh;
                rz = fmaT(rh, rh, rz);
                rr = fmaT(c.D[i] * rh, rh, rr);
                return;
            }
            const T ri = bi - ax;
            V.r[i] = ri;
            rr = fmaT(ri, ri, rr);
            if (V.z) {
                const T zi = V.dinv[i] * ri;
                V.z[i] = zi;
                rz = fmaT(ri, zi, rz);
            }
        });
    }
    // p at global cell (gx, gy, z), 0 outside the grid
    __device__ __forceinline__ T pat(const Vecs<T> &V, const T *pold, bool first, T beta, int gx, int gy,
                                     int z) const {
        if (z < 0 || z >= s.nz || gx < 0 || gx >= s.nx || gy < 0 || gy >= s.ny) return T(0);
        const int64_t i = gx + (int64_t)s.nx * gy + (int64_t)s.nx * s.ny * z;
        const T zi = ldcg(V.z + i);
        return first ? zi : fmaT(beta, ldcg(pold + i), zi);
    }
    // p at an own cell; DX: also x += ax p_old there (the last iteration's update)
    __device__ __forceinline__ T pat_own(const Vecs<T> &V, const T *pold, bool first, T beta, T ax, int gx, int gy,
                                         int z) const {
        if constexpr (DX) {
            if (z < 0 || z >= s.nz || gx < 0 || gx >= s.nx || gy < 0 || gy >= s.ny) return T(0);
            const int64_t i = gx + (int64_t)s.nx * gy + (int64_t)s.nx * s.ny * z;
            const T zi = ldcg(V.z + i);
            if (first) return zi;
            const T po = ldcg(pold + i);
            V.x[i] = fmaT(ax, po, V.x[i]);
            return fmaT(beta, po, zi);
        } else {
            return pat(V, pold, first, beta, gx, gy, z);
        }
    }
    __device__ void flush_x(const Vecs<T> &V, const T *p, T alpha) const {
        each_cell([&](int64_t i) { V.x[i] = fmaT(alpha, p[i], V.x[i]); });
    }
    // F2D: p.q as an FP32 pair of the values scaled by 2^-ps, into pair[0..2)
    // if given, else added to pq
    __device__ void phaseA_block(const Vecs<T> &V, const T *pold, T *pout, bool first, T beta, T &pq, T *sm,
                                 int ps, float *pair = nullptr, T ax = T(0)) const {
        const int64_t nu = units();
        float fh = 0.f, fl = 0.f;
        for (int64_t u = blockIdx.x; u < nu; u += gridDim.x)
            phaseA_unit(u, V, pold, pout, first, beta, pq, sm, ps, fh, fl, ax);
        if constexpr (F2D) {
            if (pair) { pair[0] = fh; pair[1] = fl; }
            else pq += f2_value(fh, fl, ps);
        }
    }
    // 2.5D march: thread (lx, ly) owns column (x, y) and keeps p at z-1, z,
    // z+1 in registers; the first kHalo threads own one cell of the plane's
    // halo ring each.  Per plane: publish plane z (own cell and ring cell) to
    // shared memory, one barrier, form q at plane z; two plane buffers
    // alternate.  Software pipeline, one plane ahead: while plane z is
    // formed, the loads that planes z+1 and z+2 need are already in flight
    // -- the coefficients of plane z+1, z and p_old (and x) of the own
    // column at z+2 and of the ring cell at z+1 -- and the arithmetic on
    // them (p = z + beta p_old, the lazy x update) happens one plane later,
    // so no load is waited for in the plane that issued it.
    static constexpr int kEx = kTileX + 2, kEy = kTileY + 2, kPls = kEx * kEy;
    static constexpr int kHalo = kPls - kTileX * kTileY;   // 84 ring cells
    __device__ __forceinline__ void halo_cell(int k, int &hx, int &hy) const {
        // ring of the (kTileX+2) x (kTileY+2) plane: bottom row, top row, left and right columns
        if (k < kEx) { hx = k; hy = 0; }
        else if (k < 2 * kEx) { hx = k - kEx; hy = kEy - 1; }
        else if (k < 2 * kEx + kTileY) { hx = 0; hy = 1 + (k - 2 * kEx); }
        else { hx = kEx - 1; hy = 1 + (k - 2 * kEx - kTileY); }
    }
    // the face coefficients of cell i at plane z (tzm comes from the plane below)
    struct Faces { T d, tym, txm, txp, typ, tzp; };
    __device__ __forceinline__ void load_faces(int64_t i, int xx, int yy, int z, Faces &f) const {
        f.d = (!UNIT) ? c.D[i] : T(0);
        f.tym = yy > 0 ? c.Ty[i - s.nx] : T(0);
        f.txm = xx > 0 ? c.Tx[i - 1] : T(0);
        f.txp = xx + 1 < s.nx ? c.Tx[i] : T(0);
        f.typ = yy + 1 < s.ny ? c.Ty[i] : T(0);
        f.tzp = z + 1 < s.nz ? c.Tz[i] : T(0);
    }
    // FP32 faces of the next plane are held in registers; FP64 ones would
    // cost ten more registers, so the FP64 march only asks L1 for their
    // lines a plane ahead and loads them in their own plane
    static constexpr bool kFacesAhead = sizeof(T) == 4;
    __device__ __forceinline__ void prefetch_faces(int64_t i, int xx, int yy, int z) const {
        const auto pf = [](const T *a) { asm volatile("prefetch.global.L1 [%0];" ::"l"(a)); };
        if (!UNIT) pf(c.D + i);
        if (yy > 0) pf(c.Ty + i - s.nx);
        if (xx > 0 && (xx & 15) == 0) pf(c.Tx + i - 1);   // other lanes' lines are those of Tx + i
        pf(c.Tx + i);
        pf(c.Ty + i);
        if (z + 1 < s.nz) pf(c.Tz + i);
    }
    __device__ void phaseA_unit(int64_t u, const Vecs<T> &V, const T *pold, T *pout, bool first, T beta, T &pq,
                                T *sm, int ps, float &fh, float &fl, T ax) const {
        int x0, y0, z0;
        origin(u, x0, y0, z0);
        const int lx = threadIdx.x % kTileX, ly = threadIdx.x / kTileX;
        const int xx = x0 + lx, yy = y0 + ly;
        const bool act = xx < s.nx && yy < s.ny;
        const int z1 = min(z0 + kTileZ, s.nz);
        const int64_t sxy = (int64_t)s.nx * s.ny;
        const bool has_h = threadIdx.x < kHalo;
        int hx = 0, hy = 0;
        if (has_h) halo_cell(threadIdx.x, hx, hy);
        const int ghx = x0 - 1 + hx, ghy = y0 - 1 + hy;
        const bool hin = has_h && ghx >= 0 && ghx < s.nx && ghy >= 0 && ghy < s.ny;
        const int cc = (ly + 1) * kEx + (lx + 1);
        const int64_t col = act ? xx + (int64_t)s.nx * yy : 0;
        const int64_t hcol = hin ? ghx + (int64_t)s.nx * ghy : 0;
        const auto mkp = [&](T zv, T pv) { return first ? zv : fmaT(beta, pv, zv); };
        // raw values of the own column one plane ahead of pn and of the ring cell at the next plane
        T oz = T(0), op = T(0), ox = T(0), hz = T(0), hp = T(0);
        T pm = T(0), pc = T(0), tzm = T(0);
        Faces cur{}, nxt{};
        // prologue: p at z0-1 and z0 (with the lazy x update at z0), raw
        // values at z0+1 (own) and z0 (ring), coefficients of plane z0
        if (act) {
            if (z0 > 0) {
                const int64_t i = col + sxy * (z0 - 1);
                pm = mkp(ldcg(V.z + i), first ? T(0) : ldcg(pold + i));
                tzm = c.Tz[i];
            }
            const int64_t i = col + sxy * z0;
            if (kFacesAhead) load_faces(i, xx, yy, z0, cur);
            else prefetch_faces(i, xx, yy, z0);
            const T zv = ldcg(V.z + i), pv = first ? T(0) : ldcg(pold + i);
            if (z0 + 1 < s.nz) {
                const int64_t j = i + sxy;
                oz = ldcg(V.z + j);
                if (!first) op = ldcg(pold + j);
                if (DX && !first && z0 + 1 < z1) ox = V.x[j];
            }
            if constexpr (DX) {
                if (!first) V.x[i] = fmaT(ax, pv, V.x[i]);
            }
            pc = mkp(zv, pv);
        }
        if (hin) {
            const int64_t i = hcol + sxy * z0;
            hz = ldcg(V.z + i);
            if (!first) hp = ldcg(pold + i);
        }
        for (int z = z0; z < z1; ++z) {
            // p of the own column at z+1 (the lazy x update there if the cell is
            // the tile's) and of the ring cell at z, from values loaded a plane ago
            T pn = T(0), ph = T(0);
            if (act && z + 1 < s.nz) {
                pn = mkp(oz, op);
                if constexpr (DX) {
                    if (!first && z + 1 < z1) V.x[col + sxy * (z + 1)] = fmaT(ax, op, ox);
                }
            }
            if (hin) ph = mkp(hz, hp);
            // loads for the next plane: coefficients of z+1, own column at z+2, ring at z+1
            if (act) {
                if constexpr (kFacesAhead) {
                    if (z + 1 < z1) load_faces(col + sxy * (z + 1), xx, yy, z + 1, nxt);
                } else {
                    load_faces(col + sxy * z, xx, yy, z, cur);   // lines asked for a plane ago
                    if (z + 1 < z1) prefetch_faces(col + sxy * (z + 1), xx, yy, z + 1);
                }
                oz = op = ox = T(0);
                if (z + 2 < s.nz && z + 2 <= z1) {
                    const int64_t j = col + sxy * (z + 2);
                    oz = ldcg(V.z + j);
                    if (!first) op = ldcg(pold + j);
                    if (DX && !first && z + 2 < z1) ox = V.x[j];
                }
            }
            if (hin && z + 1 < z1) {
                const int64_t j = hcol + sxy * (z + 1);
                hz = ldcg(V.z + j);
                if (!first) hp = ldcg(pold + j);
            }
            T *pl = sm + (z & 1) * kPls;
            pl[cc] = pc;
            if (has_h) pl[hy * kEx + hx] = ph;
            __syncthreads();
            if (act) {
                const int64_t i = col + sxy * z;
                T qi = UNIT ? pc : cur.d * pc;
                qi = fmaT(-tzm, pm, qi);
                qi = fmaT(-cur.tym, pl[cc - kEx], qi);
                qi = fmaT(-cur.txm, pl[cc - 1], qi);
                qi = fmaT(-cur.txp, pl[cc + 1], qi);
                qi = fmaT(-cur.typ, pl[cc + kEx], qi);
                qi = fmaT(-cur.tzp, pn, qi);
                pout[i] = pc;
                V.q[i] = qi;
                if constexpr (F2D) {
                    float ph_, pl_, qh_, ql_;
                    split_f2((double)pc, ps, ph_, pl_);
                    split_f2((double)qi, ps, qh_, ql_);
                    f2_add_prod(ph_, pl_, qh_, ql_, fh, fl);
                } else {
                    pq = fmaT(pc, qi, pq);
                }
            }
            pm = pc;
            pc = pn;
            tzm = cur.tzp;
            if constexpr (kFacesAhead) cur = nxt;
        }
        __syncthreads();
    }
};

// CSR: one row per thread; the p of every referenced column is recomputed
// from z and p_old (rows are independent, no shared memory).
// SP (store p): phase A first forms p = z + beta p_old once per row and
// stores it, then -- after a grid barrier -- the product reads p at the
// columns: one FP64 FMA and one load per entry instead of two of each, for
// one barrier more per iteration (large global systems, where the
// recomputation's FP64 work and L2 loads bound the iteration).
template <typename T, bool SP = false>
struct OpCsr {
    Csr cs;
    const T *av;
    int32_t n;   // resolved at kernel start (device-side count of an extracted subsystem)
    const int32_t *done = nullptr;   // set: the cluster kernel may have solved the system already
    Ctrl *bar = nullptr;             // SP: the control block of the launch's grid barrier
    static constexpr int kSmem = 1;
    static constexpr bool kAnyBlock = true;    // rows dealt to warps: any block size
    static constexpr bool kScaled = false;
    static constexpr bool kPairDots = sizeof(T) == 8;   // FP64: block sums on FP32 pairs
    static constexpr bool kDeferX = false;
    __device__ bool skipped() const { return done && *done; }
    __device__ void resolve() { if (cs.n_dev) n = *cs.n_dev; }
    __device__ void prologue(const Vecs<T> &) const {}
    __device__ void epilogue(const Vecs<T> &) const {}
    __device__ void zero_solution(const Vecs<T> &V) const { each_cell([&](int64_t i) { V.x[i] = T(0); }); }
    __device__ void phaseB_block(const Vecs<T> &V, const T *p, T alpha, T (&acc)[2], int) const {
        phaseB_generic(*this, V, p, alpha, acc);
    }
    // Extracted subsystems (row count on the device): rows dealt to warps
    // across blocks -- global warp g = warp * gridDim.x + block takes rows
    // 32 g .. 32 g + 31, then the same plus all threads -- so a small system
    // spreads over every SM instead of filling the first blocks.  Other
    // systems: consecutive rows per block.
    template <class F>
    __device__ __forceinline__ void each_cell(F f) const {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const int64_t i0 = cs.n_dev ? ((int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31)
                                    : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (int64_t i = i0; i < n; i += stride) f(i);
    }
    __device__ void setup_block(const Vecs<T> &V, T &bb, T &rz, T &rr) const {
        each_cell([&](int64_t i) {
            T ax = T(0);
            const int32_t e1 = cs.rp[i + 1];
            for (int32_t e = cs.rp[i]; e < e1; ++e) ax = fmaT(av[e], ldcg(V.x + LC_IDX(cs.ci[e], n)), ax);
            const T bi = V.b[i];
            const T ri = bi - ax;
            V.r[i] = ri;
            bb = fmaT(bi, bi, bb);
            rr = fmaT(ri, ri, rr);
            if (V.z) {
                const T zi = V.dinv[i] * ri;
                V.z[i] = zi;
                rz = fmaT(ri, zi, rz);
            }
        });
    }
    // pair (FP64): the thread's p.q split into an FP32 pair scaled by 2^-2 ps
    __device__ void phaseA_block(const Vecs<T> &V, const T *pold, T *pout, bool first, T beta, T &pq, T *,
                                 int ps, float *pair = nullptr, T = T(0)) const {
        if constexpr (SP) {
            // own rows: z and p_old were written by this thread (the same row mapping in every phase)
            each_cell([&](int64_t i) {
                const T zi = V.z[i];
                pout[i] = first ? zi : fmaT(beta, pold[i], zi);
            });
            grid_sync(bar, gridDim.x);   // a timeout is recorded; the next reduction's wait ends the solve
            each_cell([&](int64_t i) {
                T qi = T(0), pi = T(0);
                const int32_t e1 = cs.rp[i + 1];
                for (int32_t e = cs.rp[i]; e < e1; ++e) {
                    const int32_t j = LC_IDX(cs.ci[e], n);
                    const T pj = ldcg(pout + j);
                    if (j == i) pi = pj;
                    qi = fmaT(av[e], pj, qi);
                }
                V.q[i] = qi;
                pq = fmaT(pi, qi, pq);
            });
        } else {
            each_cell([&](int64_t i) {
                T qi = T(0), pi = T(0);
                const int32_t e1 = cs.rp[i + 1];
                for (int32_t e = cs.rp[i]; e < e1; ++e) {
                    const int32_t j = LC_IDX(cs.ci[e], n);
                    const T zj = ldcg(V.z + j);
                    const T pj = first ? zj : fmaT(beta, ldcg(pold + j), zj);
                    if (j == i) pi = pj;
                    qi = fmaT(av[e], pj, qi);
                }
                pout[i] = pi;
                V.q[i] = qi;
                pq = fmaT(pi, qi, pq);
            });
        }
        if constexpr (kPairDots)
            if (pair) split_f2((double)pq, 2 * ps, pair[0], pair[1]);
    }
};

// -------------------------------------------------------------- building blocks

// r = b - A x (z = dinv r if V.z), with the grid sums of b.b, r.z, r.r.
template <class OP, typename T>
__device__ bool residual_phase(const OP &op, const Vecs<T> &V, double *part, double *red, Ctrl *ctrl, double &bb,
                               double &rz, double &rr) {
    T acc[3] = {T(0), T(0), T(0)};
    op.setup_block(V, acc[0], acc[1], acc[2]);
    double out[3];
    if (!grid_sums<3, 0, T>(acc, 0, part, red, ctrl, out)) return false;
    bb = out[0];
    rz = out[1];
    rr = out[2];
    return true;
}

// CG iterations from the current r, z (first phase with p = z).  Stops when
// r.r <= stop on the recurrence residual, at maxit, or on breakdown.
// Returns 1 converged, 0 iteration limit, -1 breakdown, -2 wait timed out.
template <class OP, typename T>
__device__ int cg_iterations(const OP &op, const Vecs<T> &V, double *part, double *red, T *sm, Ctrl *ctrl,
                             double rz, double stop, int maxit, int &it, int &pin, int nscale = 0,
                             double rr = 0.0) {
    bool first = true;
    double beta = 0.0;
    double rrp = rr;   // last r.r total (unscaled ops with pair sums: the scale of the next)
    double alpha_x = 0.0;   // kDeferX: the alpha whose x update rides on the next phase A
    while (true) {
        T pq = T(0);
        const T *pold = pin ? V.p1 : V.p0;
        T *pout = pin ? V.p0 : V.p1;
        double o1[3];   // p.q, alpha, breakdown flag
        const double rz_ = rz;
        const auto post1 = [rz_](double *t) {
            const bool ok = t[0] > 0.0 && isfinite(t[0]);
            t[1] = ok ? rz_ / t[0] : 0.0;
            t[2] = ok ? 0.0 : 1.0;
        };
        // pair dots: values scaled by 2^-ps, ps half the exponent of r.z, so
        // that the scaled sums stay near 1 whatever the residual's size
        const int ps = ((int)((__double_as_longlong(rz) >> 52) & 0x7ff) - 1023) >> 1;
        if constexpr (OP::kPairDots) {
            float pr[2] = {0.f, 0.f};
            op.phaseA_block(V, pold, pout, first, (T)beta, pq, sm, ps, pr, (T)alpha_x);
            const float h1[1] = {pr[0]}, l1[1] = {pr[1]};
            const int e1[1] = {2 * ps};
            if (!grid_sums_pair<1, 2>(h1, l1, e1, 3, part, red, ctrl, o1, post1)) return -2;
        } else {
            op.phaseA_block(V, pold, pout, first, (T)beta, pq, sm, nscale, nullptr, (T)alpha_x);
            T a1[1] = {pq};
            if (!grid_sums<1, 2, T>(a1, 3, part, red, ctrl, o1, post1)) return -2;
        }
        if (flag_set(o1[2])) return -1;
        const T alpha = (T)o1[1];
        pin ^= 1;
        const T *p = pout;
        T acc[2] = {T(0), T(0)};
        op.phaseB_block(V, p, alpha, acc, nscale);
        double o2[4];   // r.z, stopping norm, converged flag, beta
        const auto post2 = [rz_, stop](double *t) {
            t[2] = t[1] <= stop ? 1.0 : 0.0;
            t[3] = t[0] / rz_;
        };
        if constexpr (OP::kPairDots) {   // r.z split into a pair; the scaled ops' FP32 norm as it is
            float h2[2], l2[2] = {0.f, 0.f};
            int e2[2] = {2 * ps, 0};
            split_f2((double)acc[0], 2 * ps, h2[0], l2[0]);
            if constexpr (OP::kScaled) {
                h2[1] = (float)acc[1];
            } else {   // r.r in FP64, scaled by its own last total
                const int pr = ((int)((__double_as_longlong(rrp) >> 52) & 0x7ff) - 1023) >> 1;
                split_f2((double)acc[1], 2 * pr, h2[1], l2[1]);
                e2[1] = 2 * pr;
            }
            if (!grid_sums_pair<2, 2>(h2, l2, e2, 4, part, red, ctrl, o2, post2)) return -2;
            rrp = o2[1];
        } else {
            if (!grid_sums<2, 2, T>(acc, 4, part, red, ctrl, o2, post2)) return -2;
        }
        ++it;
        const bool conv = flag_set(o2[2]);
        if (conv || it >= maxit) {
            if constexpr (OP::kDeferX) {   // the pending x += alpha p, before anyone reads x
                op.flush_x(V, p, alpha);
                if (!grid_sync(ctrl, gridDim.x)) return -2;
            }
            return conv ? 1 : 0;
        }
        beta = o2[3];
        rz = o2[0];
        first = false;
        alpha_x = (double)alpha;
    }
}

// -------------------------------------------------------------- kernels

template <class OP, int MINB, int THREADS = kPcgThreads>
__global__ void __launch_bounds__(THREADS, MINB) pcg_kernel(OP op, Vecs<double> V, double *part, double tol,
                                                            int maxit, int max_restarts, Ctrl *ctrl) {
    __shared__ double red[128];
    __shared__ __align__(16) double sm[OP::kSmem];
    if (op.skipped()) return;
    op.resolve();
    if (OP::kScaled) {   // x^ = D^1/2 x into the workspace (the caller's x stays untouched until the end)
        op.prologue(V);
        if (!grid_sync(ctrl, gridDim.x)) return;
    }
    double bb, rz, rr;
    if (!residual_phase(op, V, part, red, ctrl, bb, rz, rr)) return;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const double stop = (tol * tol) * bb;
    if (lead) {
        ctrl->bnorm2 = bb;
        ctrl->relres0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    if (bb == 0.0) {   // A x = 0: x = 0
        op.zero_solution(V);
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = 0.0; }
        return;
    }
    if (rr <= stop) {   // the starting iterate is returned as it is
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = sqrt(rr / bb); }
        return;
    }
    // scaled solves sum the stopping norm sum D r^^2 in FP32, relative to
    // 2^(2 e) ~ b.b: D 2^-2h times (|r^| 2^-(e-h))^2
    int nscale = 0;
    double stop_rec = stop;
    if constexpr (OP::kScaled) {
        const int e = (((int)((__double_as_longlong(bb) >> 52) & 0x7ff)) - 1023) >> 1;
        nscale = e - op.dn_shift();
        stop_rec = ldexp(stop, -2 * e);
    }
    int it = 0, restarts = 0, pin = 0, result;
    while (true) {
        result = cg_iterations(op, V, part, red, sm, ctrl, rz, stop_rec, maxit, it, pin, nscale, rr);
        if (result == -2) return;
        if (result != 1) break;
        // converged on the recurrence residual: confirm with the true one
        double bb2;
        if (!residual_phase(op, V, part, red, ctrl, bb2, rz, rr)) return;
        if (rr <= stop) break;
        result = 0;
        if (++restarts > max_restarts || it >= maxit) break;
    }
    if (result == 0 && it >= maxit) {   // report the true residual of the last iterate
        double bb2, rz2;
        if (!residual_phase(op, V, part, red, ctrl, bb2, rz2, rr)) return;
    }
    op.epilogue(V);   // scaled solves: x = D^-1/2 x^
    if (lead) {
        ctrl->iters = it;
        ctrl->restarts = restarts;
        ctrl->converged = result;
        ctrl->early = 0;
        ctrl->relres = sqrt(rr / bb);
        if (result == -1) atomicCAS(&ctrl->status, LC_OK, LC_ERR_BREAKDOWN);
    }
}

// Iterative refinement: FP64 residual and update around FP32 inner CG.
template <class OPD, class OPF, int MINB, int THREADS = kPcgThreads>
__global__ void __launch_bounds__(THREADS, MINB) ir_kernel(OPD opd, OPF opf, Vecs<double> VD, Vecs<float> VF,
                                                           double *part, double tol, double inner_tol,
                                                           int maxit, int max_outer, Ctrl *ctrl) {
    __shared__ double red[128];
    __shared__ __align__(16) float sm[OPF::kSmem];
    opd.resolve();
    opf.resolve();
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    int it = 0, outer = 0, result = 0, pin = 0;
    double bb = 0.0, rr = 0.0, stop = 0.0;
    while (true) {
        // FP64 residual r = b - A x (no z)
        double bbo, rzo;
        if (!residual_phase(opd, VD, part, red, ctrl, bbo, rzo, rr)) return;
        if (outer == 0) {
            bb = bbo;
            stop = (tol * tol) * bb;
            if (lead) {
                ctrl->bnorm2 = bb;
                ctrl->relres0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
            }
            if (bb == 0.0) {
                opd.each_cell([&](int64_t i) { VD.x[i] = 0.0; });
                if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = 0.0; }
                return;
            }
        }
        if (rr <= stop) { result = 1; break; }
        if (outer >= max_outer || it >= maxit) { result = 0; break; }
        // inner problem: fl32(A) d = fl32(r / ||r||), d = 0; on the scaled
        // operator S fl32(A) S d^ = fl32(S r / ||r||), d = S d^
        const double sc = sqrt(rr), inv = 1.0 / sc;
        float acc[2] = {0.f, 0.f};
        opf.each_cell([&](int64_t i) {
            if constexpr (OPF::kScaled) {
                const float ri = (float)(opf.sc[i] * ldcg(VD.r + i) * inv);
                const float t = opf.d32[i] * ri;
                VF.r[i] = ri;
                VF.x[i] = 0.f;
                acc[0] = fmaf(ri, ri, acc[0]);
                acc[1] = fmaf(t, t, acc[1]);
            } else {
                const float ri = (float)(ldcg(VD.r + i) * inv);
                const float zi = VF.dinv[i] * ri;
                VF.r[i] = ri;
                VF.z[i] = zi;
                VF.x[i] = 0.f;
                acc[0] = fmaf(ri, zi, acc[0]);
                acc[1] = fmaf(ri, ri, acc[1]);
            }
        });
        double o[2];
        if (!grid_sums<2, 0, float>(acc, 6, part, red, ctrl, o)) return;
        // the inner solve reduces its residual by inner_tol, or -- when less is
        // missing -- by half of what the outer test still needs (no over-solving
        // in the last sweep)
        const double need = 0.5 * sqrt(stop / rr);
        const double red_in = need > inner_tol ? need : inner_tol;
        const double stop_in = (red_in * red_in) * o[1];
        const int res = cg_iterations(opf, VF, part, red, sm, ctrl, o[0], stop_in, maxit, it, pin);
        if (res == -2) return;
        if (res == -1) { result = -1; break; }
        // x += ||r|| d in FP64
        if constexpr (OPF::kScaled)
            opd.each_cell([&](int64_t i) { VD.x[i] = fma(sc, opf.sc[i] * (double)ldcg(VF.x + i), VD.x[i]); });
        else
            opd.each_cell([&](int64_t i) { VD.x[i] = fma(sc, (double)ldcg(VF.x + i), VD.x[i]); });
        ++outer;
        if (!grid_sync(ctrl, gridDim.x)) return;
    }
    if (lead) {
        ctrl->iters = it;
        ctrl->restarts = outer;
        ctrl->outer = outer;
        ctrl->converged = result;
        ctrl->early = (result == 1 && outer == 0) ? 1 : 0;
        ctrl->relres = sqrt(rr / bb);
        if (result == -1) atomicCAS(&ctrl->status, LC_OK, LC_ERR_BREAKDOWN);
    }
}

// -------------------------------------------------------------- small kernels

template <typename T>
__global__ void csr_dinv_kernel(Csr c, const T *av, T *dinv) {
    const int32_t n = c.n_dev ? *c.n_dev : c.n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T d = T(0);
        const int32_t e1 = c.rp[i + 1];
        for (int32_t e = c.rp[i]; e < e1; ++e)
            if (c.ci[e] == i) d = av[e];
        dinv[i] = T(1) / d;
    }
}

// FP32 copy of the CSR values (of the first *n_dev rows, or all rows).
__global__ void csr_to_f32_kernel(Csr c, float *av32) {
    const int32_t n = c.n_dev ? *c.n_dev : c.n;
    const int32_t nnz = c.rp[n];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        av32[e] = (float)c.av[e];
}

__global__ void reset_ctrl_kernel(Ctrl *ctrl) {
    ctrl->bar_count = 0;
    ctrl->iters = 0;
    ctrl->restarts = 0;
    ctrl->outer = 0;
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

// -------------------------------------------------------------- launch

int coop_grid(const void *kernel, int64_t units, int cap, int threads = kPcgThreads) {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
    int64_t g = (int64_t)sms * (per < 1 ? 1 : per);
    if (cap > 0 && g > cap) g = cap;
    if (g > units) g = units;
    if (g > kMaxGrid) g = kMaxGrid;
    return (int)(g < 1 ? 1 : g);
}

// minblocks = the register budget asked of the compiler (blocks of 256
// threads that must fit on one SM): 1 = unconstrained, 2..4 = at most
// 128 / 85 / 64 registers per thread.  big: one block of kBigThreads per SM
// instead (operators with per-warp work only): the register budget of three
// blocks of 256, a third of the block partials and barrier arrivals per
// grid reduction.
constexpr int kBigThreads = 768;

template <class OP>
const void *pcg_kernel_for(int minblocks, bool big) {
    if constexpr (OP::kAnyBlock)
        if (big) return (const void *)pcg_kernel<OP, 1, kBigThreads>;
    switch (minblocks) {
        case 2: return (const void *)pcg_kernel<OP, 2>;
        case 3: return (const void *)pcg_kernel<OP, 3>;
        case 4: return (const void *)pcg_kernel<OP, 4>;
        default: return (const void *)pcg_kernel<OP, 1>;
    }
}
template <class OPD, class OPF>
const void *ir_kernel_for(int minblocks, bool big) {
    if constexpr (OPD::kAnyBlock && OPF::kAnyBlock)
        if (big) return (const void *)ir_kernel<OPD, OPF, 1, kBigThreads>;
    switch (minblocks) {
        case 2: return (const void *)ir_kernel<OPD, OPF, 2>;
        case 3: return (const void *)ir_kernel<OPD, OPF, 3>;
        case 4: return (const void *)ir_kernel<OPD, OPF, 4>;
        default: return (const void *)ir_kernel<OPD, OPF, 1>;
    }
}

cudaError_t coop_launch(const void *k, int64_t units, int cap, void **args, Ctrl *ctrl, cudaStream_t s,
                        bool reset = true, int threads = kPcgThreads) {
    const int grid = coop_grid(k, units, cap, threads);
    if (reset) {
        reset_ctrl_kernel<<<1, 1, 0, s>>>(ctrl);
        note_launches(1);
    }
    note_launches(1);
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(threads), args, 0, s);
}

template <class OP>
cudaError_t launch_pcg(const OP &op, int64_t units, const Vecs<double> &V, double *part, const PcgArgs &a,
                       Ctrl *ctrl, int cap, int minblocks, cudaStream_t s, bool reset = true) {
    OP o = op;
    Vecs<double> v = V;
    double *pt = part;
    double t = a.tol;
    int mi = a.maxit, mr = a.max_restarts;
    Ctrl *c = ctrl;
    void *args[] = {&o, &v, &pt, &t, &mi, &mr, &c};
    const bool big = a.big && OP::kAnyBlock;
    const int threads = big ? kBigThreads : kPcgThreads;
    // units counts blocks of kPcgThreads: the same warps in fewer, larger blocks
    const int64_t ub = (units * kPcgThreads + threads - 1) / threads;
    return coop_launch(pcg_kernel_for<OP>(minblocks, big), ub, cap, args, ctrl, s, reset, threads);
}

template <class OPD, class OPF>
cudaError_t launch_ir(const OPD &opd, const OPF &opf, int64_t units, const Vecs<double> &VD, const Vecs<float> &VF,
                      double *part, const PcgArgs &a, Ctrl *ctrl, int cap, int minblocks, cudaStream_t s) {
    OPD od = opd;
    OPF of = opf;
    Vecs<double> vd = VD;
    Vecs<float> vf = VF;
    double *pt = part;
    double t = a.tol, ti = a.inner_tol;
    int mi = a.maxit, mo = a.max_outer;
    Ctrl *c = ctrl;
    void *args[] = {&od, &of, &vd, &vf, &pt, &t, &ti, &mi, &mo, &c};
    const bool big = a.big && OPD::kAnyBlock && OPF::kAnyBlock;
    const int threads = big ? kBigThreads : kPcgThreads;
    const int64_t ub = (units * kPcgThreads + threads - 1) / threads;
    return coop_launch(ir_kernel_for<OPD, OPF>(minblocks, big), ub, cap, args, ctrl, s, true, threads);
}

Vecs<double> vecs64(const PcgArgs &a, const PcgWork &w, const double *dinv) {
    Vecs<double> V;
    V.b = a.b; V.x = a.x; V.r = w.r; V.z = w.z; V.q = w.q; V.p0 = w.p0; V.p1 = w.p1; V.dinv = dinv;
    V.xu = nullptr;
    return V;
}
Vecs<float> vecs32(const PcgWork &w, const float *dinv32) {
    Vecs<float> V;
    V.b = nullptr; V.x = w.x32; V.r = w.r32; V.z = w.z32; V.q = w.q32; V.p0 = w.p032; V.p1 = w.p132; V.dinv = dinv32;
    V.xu = nullptr;
    return V;
}

Coef<double> coef64(const Stencil &s) { return {s.D, s.Tx, s.Ty, s.Tz}; }
Coef<float> coef32(const Stencil &s) { return {s.D32, s.Tx32, s.Ty32, s.Tz32}; }

}  // namespace

}  // namespace lc
