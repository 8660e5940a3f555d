// lc_pcgpipe.cu -- pipelined Jacobi-PCG (the Ghysels-Vanroose arrangement)
// for CSR systems whose solve is bound by latency and FP64 issue: the
// extracted local subsystem of Alg 1 (step 5).  One grid barrier per
// iteration, the iteration's grid sums read while the matrix-vector product
// runs, and the symmetrically scaled system so that the Jacobi
// preconditioner is the identity.
//
// Jacobi-PCG on B x = b is CG on the scaled system  Bh xh = bh  with
// S = diag(B)^-1/2, Bh = S B S (unit diagonal), bh = S b, x = S xh: the same
// iterates in exact arithmetic, and the unscaled residual is r = S^-1 rh.
// CG in the pipelined arrangement, w = Bh r carried along by recurrence:
//   gamma_i = (r_i, r_i),  delta_i = (w_i, r_i),  n_i = Bh w_i
//   beta_i = gamma_i / gamma_(i-1),  alpha_i = gamma_i / (delta_i - beta_i gamma_i / alpha_(i-1))
//   z_i = n_i + beta_i z_(i-1)  (= Bh s_i),  s_i = w_i + beta_i s_(i-1)  (= Bh p_i),
//   p_i = r_i + beta_i p_(i-1)
//   x_(i+1) = x_i + alpha_i p_i,  r_(i+1) = r_i - alpha_i s_i,  w_(i+1) = w_i - alpha_i z_i
// The stopping norm ||r||^2 = sum_i d_i rh_i^2 is summed in FP32, rh_i scaled
// by 2^-e with 2^(2e) ~ ||b||^2 to stay in FP32's range (approx_abs_f32;
// relative error ~1e-7 in a test against tol^2 ||b||^2); the true residual
// that confirms convergence is FP64.  FP64 instructions
// per row and iteration: the row's entries (one FMA each) and six vector
// updates (21 in the unscaled form); gamma and delta are summed on FP32 pairs
// (split_f2, f2_add_prod: ~2^-45 relative per term), the block sums too.
//
// Per iteration, in one persistent cooperative launch:
//   after the barrier: warp 0 of every block adds the block partials of
//     gamma, delta and the stopping norm and derives alpha, beta and the
//     stopping and breakdown flags, while the other warps form n = Bh w for
//     their rows (the neighbours' w of the previous phase);
//   block barrier; the other warps update z, s, p, x, r, w of their rows and
//     form the partials of the next sums; block sums; grid barrier.
// w is double-buffered (neighbours read it in the product while its owner
// writes the next one); z, s, p, x, r, n are touched by their owner only.
// The partial slots alternate between two sets: a block may write the next
// partials while a slower one still reads these.  Stopping test,
// true-residual confirmation and restarts follow the two-reduction kernel
// (lc_pcg_impl.cuh), with the same Ctrl fields.
//
// pcgpipe_mix_kernel (mixed precision, below) runs the same arrangement in
// FP32 as the inner solve of FP64 iterative refinement.
#include "lc_pcg_impl.cuh"

namespace lc {

namespace {

constexpr int kPipeThreads = 512;              // one block per SM (no register spills; 768: 80 registers, spills)
constexpr int kPipeWarps = kPipeThreads / 32;  // warp 0 reduces, the others take rows

struct PipeArgs {
    Csr cs;                  // B (rows and columns of the subsystem)
    const double *b;
    double *x;
    double *ah;              // Bh values, B's pattern (formed by the kernel)
    double *sd;              // S = diag(B)^-1/2 (formed by the kernel)
    float *d32;              // fl32(diag(B)) (formed by the kernel)
    double *xh;              // S^-1 x (the iterate)
    double *r, *w[2], *z, *s, *p, *n;
    double *part;
    double tol;
    int maxit, max_restarts;
    Ctrl *ctrl;
    const int32_t *done;   // set: a cluster kernel launched before may already have solved it
};

__global__ void pipe_reset_kernel(Ctrl *ctrl) {
    ctrl->bar_count = 0;
    ctrl->iters = 0;
    ctrl->restarts = 0;
    ctrl->outer = 0;
    ctrl->converged = 0;
    ctrl->early = 0;
}

// Rows of this thread: warps 1.. of every block, dealt across blocks (global
// row warp g = (warp - 1) x blocks + block takes rows 32 g .. 32 g + 31, then
// every 32 G rows, G = (kPipeWarps - 1) x blocks), so a small system spreads
// over all SMs.
struct Rows {
    int64_t first, step;
    __device__ Rows() {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int64_t g = (int64_t)(warp - 1) * gridDim.x + blockIdx.x;
        first = warp == 0 ? INT64_MAX : 32 * g + lane;
        step = 32 * (int64_t)(kPipeWarps - 1) * gridDim.x;
    }
};

// (Bh v)_i in the row's entry order; v of other rows through L2
__device__ __forceinline__ double row_av(const Csr &cs, const double *__restrict__ ah, const double *v, int32_t n,
                                         int64_t i) {
    double acc = 0.0;
    const int32_t e1 = cs.rp[i + 1];
    for (int32_t e = cs.rp[i]; e < e1; ++e) acc = fma(ah[e], ldcg(v + LC_IDX(cs.ci[e], n)), acc);
    return acc;
}

// Block sums of NV values into the partial slots slot0.. (thread 0 writes),
// then the grid barrier; the totals are read later (pipe_totals).
template <int NV>
__device__ __forceinline__ bool pipe_publish(double (&v)[NV], int slot0, double *part, double *red, Ctrl *ctrl) {
    block_sum<NV, double>(v, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) part[(size_t)(slot0 + k) * kMaxGrid + blockIdx.x] = v[k];
    return grid_sync(ctrl, gridDim.x);
}

// pipe_publish for FP32 pairs: value k is (h[k] + l[k]) 2^e[k]; warps and the
// block add pairs with FP32 two-sums, thread 0 writes the block's pair.  (An FP64 warp instruction holds the FP64 pipe as long with one
// active lane as with 32, so FP64 shuffle trees over every warp of the block
// would cost about as much FP64 issue as the rows' own arithmetic.)
template <int NV>
__device__ __forceinline__ bool pipe_publish_pair(float (&h)[NV], float (&l)[NV], int slot0, double *part, double *red,
                                                  Ctrl *ctrl) {
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float bh = __shfl_down_sync(kFull, h[k], o), bl = __shfl_down_sync(kFull, l[k], o);
            pair_add(h[k], l[k], bh, bl);
        }
    // the warps' pairs into red[0..2 NV x 32) (floats): warp 0 last read them
    // before the previous grid barrier, and the step lengths live above
    float *fs = reinterpret_cast<float *>(red);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) { fs[(2 * k) * 32 + warp] = h[k]; fs[(2 * k + 1) * 32 + warp] = l[k]; }
    __syncthreads();
    // warp 0: the block's pair into its slot, then the grid barrier (as
    // grid_sync: counting arrival, bounded wait) while the other warps wait
    // at the block barrier -- two block barriers in all
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            h[k] = lane < nw ? fs[(2 * k) * 32 + lane] : 0.0f;
            l[k] = lane < nw ? fs[(2 * k + 1) * 32 + lane] : 0.0f;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const float bh = __shfl_down_sync(kFull, h[k], o), bl = __shfl_down_sync(kFull, l[k], o);
                pair_add(h[k], l[k], bh, bl);
            }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k)
                reinterpret_cast<float2 *>(part)[(size_t)(slot0 + k) * kMaxGrid + blockIdx.x] = make_float2(h[k], l[k]);
            const unsigned nb = gridDim.x;
            const unsigned long long old = atom_add_release_u64(&ctrl->bar_count, 1ull);
            const unsigned long long target = (old / nb + 1) * nb;
            int ok = 1;
            if (old + 1 < target) {
                const long long t0 = clock64();
                while (ld_acquire_u64(&ctrl->bar_count) < target) {
                    if (clock64() - t0 > kBarrierTimeoutCycles) { ok = 0; break; }
                }
            }
            if (!ok) atomicCAS(&ctrl->status, LC_OK, LC_ERR_TIMEOUT);
            s_ok = ok;
        }
        __syncwarp();
    }
    __syncthreads();
    return s_ok != 0;
}

// Warp 0: the totals of pipe_publish_pair's slots, the blocks' pairs added
// lane-strided and by a shuffle tree in a fixed order (identical in every
// block); t[k] = (h + l) 2^e[k] in FP64.
template <int NV>
__device__ __forceinline__ void pipe_totals_pair(int slot0, const double *part, const int (&e)[NV], double (&t)[NV]) {
    float h[NV], l[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) { h[k] = 0.f; l[k] = 0.f; }
    const float2 *pp = reinterpret_cast<const float2 *>(part);
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 32)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float2 v = __ldcg(pp + (size_t)(slot0 + k) * kMaxGrid + b);
            pair_add(h[k], l[k], v.x, v.y);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float bh = __shfl_down_sync(kFull, h[k], o), bl = __shfl_down_sync(kFull, l[k], o);
            pair_add(h[k], l[k], bh, bl);
        }
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] = ldexp((double)h[k] + (double)l[k], e[k]);
}

// Warp 0: the totals of slots slot0.. (after pipe_publish's barrier), lane-
// strided and reduced in a fixed order, identical in every block.
template <int NV>
__device__ __forceinline__ void pipe_totals(int slot0, const double *part, double (&t)[NV]) {
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 32)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += ldcg(part + (size_t)(slot0 + k) * kMaxGrid + b);
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] = warp_sum(acc[k]);
}

// The second half of a set-up: w = Bh rh (into w[0]) from every row's rh,
// the sums gamma, delta after a grid barrier.  With form_ah the own rows'
// Bh values are formed first (S of the neighbours is then complete).
__device__ bool pipe_setup_w(const PipeArgs &a, int32_t n, double *red, bool form_ah, double &gam, double &del) {
    const Csr &cs = a.cs;
    const Rows R;
    double acc2[2] = {0.0, 0.0};
    for (int64_t i = R.first; i < n; i += R.step) {
        double wi = 0.0;
        if (form_ah) {   // the row's Bh values, and w from them as they are formed
            const double si = a.sd[i];
            const int32_t e1 = cs.rp[i + 1];
            for (int32_t e = cs.rp[i]; e < e1; ++e) {
                const int32_t j = LC_IDX(cs.ci[e], n);
                const double v = j == i ? 1.0 : cs.av[e] * si * ldcg(a.sd + j);
                a.ah[e] = v;
                wi = fma(v, ldcg(a.r + j), wi);
            }
        } else {
            wi = row_av(cs, a.ah, a.r, n, i);
        }
        const double ri = a.r[i];
        a.w[0][i] = wi;
        acc2[0] = fma(ri, ri, acc2[0]);
        acc2[1] = fma(wi, ri, acc2[1]);
    }
    if (!pipe_publish<2>(acc2, 2, a.part, red, a.ctrl)) return false;
    double t2[2];
    if (threadIdx.x < 32) {
        pipe_totals<2>(2, a.part, t2);
        if (threadIdx.x == 0) { red[96] = t2[0]; red[97] = t2[1]; }
    }
    __syncthreads();
    gam = red[96];
    del = red[97];
    __syncthreads();
    return true;
}

// Warp 0 of every block: the totals of the two sums in slots 0, 1.
__device__ void pipe_totals2(const PipeArgs &a, double *red, double &t0, double &t1) {
    double t[2];
    if (threadIdx.x < 32) {
        pipe_totals<2>(0, a.part, t);
        if (threadIdx.x == 0) { red[96] = t[0]; red[97] = t[1]; }
    }
    __syncthreads();
    t0 = red[96];
    t1 = red[97];
    __syncthreads();
}

// The first set-up, from the unscaled system: per own row d = B_ii, S, fl32(D),
// r = b - B x (FP64, the row's entry order), rh = S r, xh = S^-1 x; the sums
// b.b and r.r; then Bh's values and w = Bh rh (pipe_setup_w).  Three grid
// barriers.
__device__ bool pipe_init(const PipeArgs &a, int32_t n, double *red, double &bb, double &rr, double &gam,
                          double &del) {
    const Csr &cs = a.cs;
    const Rows R;
    double acc[2] = {0.0, 0.0};
    for (int64_t i = R.first; i < n; i += R.step) {
        double ri = a.b[i], d = 0.0;
        const int32_t e1 = cs.rp[i + 1];
        for (int32_t e = cs.rp[i]; e < e1; ++e) {
            const int32_t j = LC_IDX(cs.ci[e], n);
            const double v = cs.av[e];
            if (j == i) d = v;
            ri = fma(-v, ldcg(a.x + j), ri);
        }
        const double q = sqrt(d), si = 1.0 / q;
        a.sd[i] = si;
        a.d32[i] = (float)d;
        a.r[i] = si * ri;
        a.xh[i] = a.x[i] * q;
        acc[0] = fma(a.b[i], a.b[i], acc[0]);
        acc[1] = fma(ri, ri, acc[1]);
    }
    if (!pipe_publish<2>(acc, 0, a.part, red, a.ctrl)) return false;
    pipe_totals2(a, red, bb, rr);
    return pipe_setup_w(a, n, red, true, gam, del);
}

// A later set-up (the true residual that confirms convergence): rh = S b - Bh
// xh, the sums b.b and ||b - B x||^2 (FP64), then w = Bh rh.
__device__ bool pipe_setup(const PipeArgs &a, int32_t n, double *red, double &bb, double &rr, double &gam,
                           double &del) {
    const Csr &cs = a.cs;
    const Rows R;
    double acc[2] = {0.0, 0.0};
    for (int64_t i = R.first; i < n; i += R.step) {
        const double si = a.sd[i], bi = a.b[i];
        const double ri = bi * si - row_av(cs, a.ah, a.xh, n, i);
        a.r[i] = ri;
        const double ru = ri / si;   // the unscaled residual
        acc[0] = fma(bi, bi, acc[0]);
        acc[1] = fma(ru, ru, acc[1]);
    }
    if (!pipe_publish<2>(acc, 0, a.part, red, a.ctrl)) return false;
    pipe_totals2(a, red, bb, rr);
    return pipe_setup_w(a, n, red, false, gam, del);
}

// Where a thread keeps the iteration state of its own rows: in the global
// vectors (any K), or, when every thread has at most kPipeRowsSm rows, in
// shared memory (row slot k of the thread at [k][thread]: r, z, s, p, xh, n,
// its own w and fl32(D)), so the row updates read nothing back from L2.
// w -- which the neighbours read -- and xh -- which the true residual after
// the iterations reads at the neighbours, right after the last grid barrier --
// are also stored to global memory every iteration.
constexpr int kPipeRowsSm = 3;
constexpr int kPipeSmVecs = 7;   // r, z, s, p, xh, n, w
constexpr size_t kPipeSmBytes = (size_t)kPipeRowsSm * kPipeThreads * (kPipeSmVecs * sizeof(double) + sizeof(float));

template <bool SM>
struct RowState {
    const PipeArgs *a;
    double *sm;    // SM: kPipeSmVecs x kPipeRowsSm x kPipeThreads doubles, then fl32(D)
    __device__ double *vec(int v, int k) const { return sm + ((size_t)v * kPipeRowsSm + k) * kPipeThreads + threadIdx.x; }
    __device__ float *d32s(int k) const {
        return reinterpret_cast<float *>(sm + (size_t)kPipeSmVecs * kPipeRowsSm * kPipeThreads) + k * kPipeThreads +
               threadIdx.x;
    }
    // v: 0 r, 1 z, 2 s, 3 p, 4 xh, 5 n
    __device__ double *gvec(int v) const {
        switch (v) {
            case 0: return a->r;
            case 1: return a->z;
            case 2: return a->s;
            case 3: return a->p;
            case 4: return a->xh;
            default: return a->n;
        }
    }
    __device__ double get(int v, int k, int64_t i) const {
        if constexpr (SM) return *vec(v, k);
        else return gvec(v)[i];
    }
    __device__ void put(int v, int k, int64_t i, double x) const {
        if constexpr (SM) *vec(v, k) = x;
        else gvec(v)[i] = x;
    }
    __device__ double w_own(int k, int64_t i, const double *wc) const {
        if constexpr (SM) return *vec(6, k);
        else return wc[i];
    }
    __device__ float d32(int k, int64_t i) const {
        if constexpr (SM) return *d32s(k);
        else return a->d32[i];
    }
};

// n = Bh w for the thread's rows when it has at most kPipeRowsSm of them: the
// rows' entries are taken in step (entry t of every row, then entry t + 1),
// so the neighbour loads of all rows are in flight together instead of one
// row's chain of column and value loads after another.  Each row still adds
// its entries in its own entry order: the same value as row_av (row_av32 in
// FP32).  G is the warp's number of row groups (the same in all its lanes),
// so a warp issues no instruction for a row group it does not have.
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T, int G>
__device__ __forceinline__ void rows_av_g(const Csr &cs, const T *__restrict__ ah, const T *v, int32_t n,
                                          const int32_t (&eb)[kPipeRowsSm], const int32_t (&ee)[kPipeRowsSm],
                                          int32_t len, T (&acc)[kPipeRowsSm]) {
    for (int32_t t = 0; t < len; ++t) {
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int32_t e = eb[k] + t;
            if (e < ee[k]) acc[k] = fma_t(ah[e], __ldcg(v + LC_IDX(cs.ci[e], n)), acc[k]);
        }
    }
}

template <typename T, class State>
__device__ __forceinline__ void rows_av_sm(const Csr &cs, const T *__restrict__ ah, const T *v, int32_t n,
                                           const Rows &R, const State &S) {
    static_assert(kPipeRowsSm == 3, "rows_av_sm takes one to three row groups");
    // a warp's 32 rows of a group are consecutive: the group exists for the
    // warp when its first row does (a ragged last group has lanes past n)
    const int64_t warp_first = R.first - (threadIdx.x & 31);
    int groups = 0;
    int32_t eb[kPipeRowsSm], ee[kPipeRowsSm];
    T acc[kPipeRowsSm];
    int32_t len = 0;
#pragma unroll
    for (int k = 0; k < kPipeRowsSm; ++k) {
        const int64_t i = R.first + k * R.step;
        acc[k] = T(0);
        eb[k] = 0;
        ee[k] = 0;
        if (warp_first + k * R.step < n) groups = k + 1;
        if (i < n) {
            eb[k] = cs.rp[i];
            ee[k] = cs.rp[i + 1];
            len = max(len, ee[k] - eb[k]);
        }
    }
    if (groups == 3) rows_av_g<T, 3>(cs, ah, v, n, eb, ee, len, acc);
    else if (groups == 2) rows_av_g<T, 2>(cs, ah, v, n, eb, ee, len, acc);
    else if (groups == 1) rows_av_g<T, 1>(cs, ah, v, n, eb, ee, len, acc);
#pragma unroll
    for (int k = 0; k < kPipeRowsSm; ++k) {
        const int64_t i = R.first + k * R.step;
        if (i < n) S.put(5, k, i, acc[k]);
    }
}

// Iterations from the state pipe_setup left (r, w[0], gamma, delta).
// Returns 1 converged, 0 iteration limit, -1 breakdown, -2 wait timed out.
template <bool SM>
__device__ int pipe_iterations(const PipeArgs &a, int32_t n, double *red, double *smem, double gam, double del,
                               double stop, int ns, int &it) {
    const Csr &cs = a.cs;
    const Rows R;
    const RowState<SM> S{&a, smem};
    if constexpr (SM) {   // the own rows' state into shared memory
        int k = 0;
        for (int64_t i = R.first; i < n; i += R.step, ++k) {
            S.put(0, k, i, a.r[i]);
            S.put(4, k, i, a.xh[i]);
            *S.vec(6, k) = a.w[0][i];
            *S.d32s(k) = a.d32[i];
        }
    }
    if (!(del > 0.0) || !isfinite(del)) return -1;
    double alpha = gam / del, beta = 0.0;
    bool first = true, pending = false;
    int cur = 0;         // w[cur] holds this iteration's w
    int pend_slot = 4;   // slots of the partials published last
    int pend_e = 0;      // their scale: gamma, delta 2^-pend_e
    int result;
    while (true) {
        // warps 1..: n = Bh w (neighbours' w of the last phase); warp 0
        // meanwhile: the totals published last and the next step lengths
        if (threadIdx.x < 32) {
            if (pending) {
                double t[3];
                const int te[3] = {pend_e, pend_e, 0};
                pipe_totals_pair<3>(pend_slot, a.part, te, t);
                if (threadIdx.x == 0) {
                    const double bt = t[0] / gam;
                    const double den = t[1] - bt * t[0] / alpha;
                    const bool ok = den > 0.0 && isfinite(den);
                    red[96] = t[0];
                    red[97] = bt;
                    red[98] = ok ? t[0] / den : 0.0;
                    red[99] = t[2] <= stop ? 1.0 : 0.0;
                    red[100] = ok ? 1.0 : 0.0;
                }
            }
        } else {
            const double *wc = a.w[cur];
            if constexpr (SM) {
                rows_av_sm(cs, a.ah, wc, n, R, S);
            } else {
                int k = 0;
                for (int64_t i = R.first; i < n; i += R.step, ++k) S.put(5, k, i, row_av(cs, a.ah, wc, n, i));
            }
        }
        __syncthreads();
        if (pending) {
            const double g1 = red[96], b1 = red[97], a1 = red[98];
            const bool conv = flag_set(red[99]), ok = flag_set(red[100]);
            if (conv) { result = 1; break; }   // (this iteration's product is not used)
            if (it >= a.maxit) { result = 0; break; }
            if (!ok) { result = -1; break; }
            gam = g1;
            beta = b1;
            alpha = a1;
            first = false;
        }
        // warps 1..: the vector updates of their rows and the next partials
        const double *wc = a.w[cur];
        double *wn = a.w[cur ^ 1];
        // gamma and delta on FP32 pairs of the values scaled by 2^-ps, ps half
        // the exponent of the last gamma
        const int ps = ((int)((__double_as_longlong(gam) >> 52) & 0x7ff) - 1023) >> 1;
        float gh = 0.f, gl = 0.f, dh = 0.f, dl = 0.f, rrf = 0.f;
        int k = 0;
        for (int64_t i = R.first; i < n; i += R.step, ++k) {
            const double ri = S.get(0, k, i), wi = S.w_own(k, i, wc), ni = S.get(5, k, i);
            double zi, si, pi;
            if (first) {
                zi = ni;
                si = wi;
                pi = ri;
            } else {
                zi = fma(beta, S.get(1, k, i), ni);
                si = fma(beta, S.get(2, k, i), wi);
                pi = fma(beta, S.get(3, k, i), ri);
            }
            const double xi = fma(alpha, pi, S.get(4, k, i));
            const double rn = fma(-alpha, si, ri);
            const double wnx = fma(-alpha, zi, wi);
            S.put(1, k, i, zi);
            S.put(2, k, i, si);
            S.put(3, k, i, pi);
            S.put(4, k, i, xi);
            S.put(0, k, i, rn);
            wn[i] = wnx;
            if constexpr (SM) {
                *S.vec(6, k) = wnx;
                a.xh[i] = xi;   // (stored, never read back: current at every grid barrier)
            }
            float rh, rl, wh, wl;
            split_f2(rn, ps, rh, rl);
            split_f2(wnx, ps, wh, wl);
            f2_add_prod(rh, rl, rh, rl, gh, gl);
            f2_add_prod(wh, wl, rh, rl, dh, dl);
            const float rf = approx_abs_f32(rn, ns);
            rrf = fmaf(S.d32(k, i) * rf, rf, rrf);
        }
        float sh[3] = {gh, dh, rrf}, sl[3] = {gl, dl, 0.f};
        pend_slot = cur ? 7 : 4;
        pend_e = 2 * ps;
        if (!pipe_publish_pair<3>(sh, sl, pend_slot, a.part, red, a.ctrl)) return -2;
        ++it;
        cur ^= 1;
        pending = true;
    }
    return result;
}

__global__ void __launch_bounds__(kPipeThreads, 1) pcgpipe_kernel(PipeArgs a) {
    __shared__ double red[128];
    extern __shared__ __align__(16) double pipe_smem[];
    if (a.done && *a.done) return;
    const int32_t n = a.cs.n_dev ? *a.cs.n_dev : a.cs.n;
    Ctrl *ctrl = a.ctrl;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const Rows R;
    double bb, rr, gam, del;
    if (!pipe_init(a, n, red, bb, rr, gam, del)) return;
    const double stop = (a.tol * a.tol) * bb;
    if (lead) {
        ctrl->bnorm2 = bb;
        ctrl->relres0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    if (bb == 0.0) {
        for (int64_t i = R.first; i < n; i += R.step) a.x[i] = 0.0;
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = 0.0; }
        return;
    }
    if (rr <= stop) {   // the starting iterate is returned as it is
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = sqrt(rr / bb); }
        return;
    }
    // the FP32 stopping norm sums (|rh| 2^-ns)^2 d with 2^(2 ns) ~ b.b
    const int ns = (((int)((__double_as_longlong(bb) >> 52) & 0x7ff)) - 1023) >> 1;
    const double stop_rec = ldexp(stop, -2 * ns);
    int it = 0, restarts = 0, result;
    while (true) {
        // the row state in shared memory when every thread has at most kPipeRowsSm rows
        result = n <= (int64_t)kPipeRowsSm * R.step
                     ? pipe_iterations<true>(a, n, red, pipe_smem, gam, del, stop_rec, ns, it)
                     : pipe_iterations<false>(a, n, red, pipe_smem, gam, del, stop_rec, ns, it);
        if (result == -2) return;
        if (result != 1) break;
        // converged on the recurrence residual: confirm with the true one
        double bb2;
        if (!pipe_setup(a, n, red, bb2, rr, gam, del)) return;
        if (rr <= stop) break;
        result = 0;
        if (++restarts > a.max_restarts || it >= a.maxit) break;
    }
    if (result == 0 && it >= a.maxit) {   // report the true residual of the last iterate
        double bb2, g2, d2;
        if (!pipe_setup(a, n, red, bb2, rr, g2, d2)) return;
    }
    for (int64_t i = R.first; i < n; i += R.step) a.x[i] = a.xh[i] * a.sd[i];
    if (lead) {
        ctrl->iters = it;
        ctrl->restarts = restarts;
        ctrl->converged = result;
        ctrl->early = 0;
        ctrl->relres = sqrt(rr / bb);
        if (result == -1) atomicCAS(&ctrl->status, LC_OK, LC_ERR_BREAKDOWN);
    }
}

// ---------------------------------------------------------------- mixed precision
//
// Iterative refinement with the pipelined CG as its FP32 inner solve (the
// deployment form with FP32 bulk iterations): the outer residual rh =
// S b - Bh xh, its norms and the update xh += sigma d stay FP64; each inner
// problem Bh d = rh / sigma (sigma = ||rh||) is solved in FP32 -- values of
// Bh rounded to FP32, every vector FP32, the sums on FP32 pairs -- from d = 0
// until its residual has dropped by inner_tol, or, when the outer test misses
// by less, by half of what is still missing.  The FP32 row state of a thread
// lives in shared memory under the same condition as the FP64 solve's.

struct PipeMixArgs {
    PipeArgs a;                 // the FP64 part: B, b, x, Bh, S, fl32(D), xh, rh (a.r)
    float *ah32;                // fl32(Bh)
    float *r, *w[2], *z, *s, *p, *n, *d;   // inner vectors (global-memory path)
    double inner_tol;
    int max_outer;
};

template <bool SM>
struct RowState32 {
    const PipeMixArgs *m;
    float *sm;   // SM: 7 x kPipeRowsSm x kPipeThreads floats
    __device__ float *vec(int v, int k) const { return sm + ((size_t)v * kPipeRowsSm + k) * kPipeThreads + threadIdx.x; }
    // v: 0 r, 1 z, 2 s, 3 p, 4 d, 5 n, 6 own w
    __device__ float *gvec(int v) const {
        switch (v) {
            case 0: return m->r;
            case 1: return m->z;
            case 2: return m->s;
            case 3: return m->p;
            case 4: return m->d;
            default: return m->n;
        }
    }
    __device__ float get(int v, int k, int64_t i) const {
        if constexpr (SM) return *vec(v, k);
        else return gvec(v)[i];
    }
    __device__ void put(int v, int k, int64_t i, float x) const {
        if constexpr (SM) *vec(v, k) = x;
        else gvec(v)[i] = x;
    }
};

__device__ __forceinline__ float row_av32(const Csr &cs, const float *__restrict__ ah, const float *v, int32_t n,
                                          int64_t i) {
    float acc = 0.f;
    const int32_t e1 = cs.rp[i + 1];
    for (int32_t e = cs.rp[i]; e < e1; ++e) acc = fmaf(ah[e], __ldcg(v + LC_IDX(cs.ci[e], n)), acc);
    return acc;
}

// One inner FP32 solve from the r (scaled, normalised), w = Bh r, gamma,
// delta left by the caller, d = 0; stops when gamma <= stop, when the FP32
// recurrences stop giving a positive step (1 in both cases), or at maxit
// inner iterations in all (0).  -1: breakdown at the start (Bh not positive
// on r: not SPD, or non-finite data); -2: a wait timed out.  d is stored to global memory every iteration (the
// caller reads it after the last grid barrier).
template <bool SM>
__device__ int pipe_inner32(const PipeMixArgs &m, int32_t n, double *red, float *smem, double gam, double del,
                            double stop, int maxit, int &it) {
    const Csr &cs = m.a.cs;
    const Rows R;
    const RowState32<SM> S{&m, smem};
    if constexpr (SM) {
        int k = 0;
        for (int64_t i = R.first; i < n; i += R.step, ++k) {
            S.put(0, k, i, m.r[i]);
            S.put(4, k, i, 0.f);
            *S.vec(6, k) = m.w[0][i];
        }
    }
    if (!(del > 0.0) || !isfinite(del)) return -1;
    double alpha = gam / del, beta = 0.0;
    bool first = true, pending = false;
    int cur = 0, pend_slot = 4, result;
    while (true) {
        if (threadIdx.x < 32) {
            if (pending) {
                double t[2];
                const int te[2] = {0, 0};
                pipe_totals_pair<2>(pend_slot, m.a.part, te, t);
                if (threadIdx.x == 0) {
                    const double bt = t[0] / gam;
                    const double den = t[1] - bt * t[0] / alpha;
                    const bool ok = den > 0.0 && isfinite(den);
                    red[96] = t[0];
                    red[97] = bt;
                    red[98] = ok ? t[0] / den : 0.0;
                    red[99] = t[0] <= stop ? 1.0 : 0.0;
                    red[100] = ok ? 1.0 : 0.0;
                }
            }
        } else {
            const float *wc = m.w[cur];
            if constexpr (SM) {
                rows_av_sm(cs, m.ah32, wc, n, R, S);
            } else {
                int k = 0;
                for (int64_t i = R.first; i < n; i += R.step, ++k) S.put(5, k, i, row_av32(cs, m.ah32, wc, n, i));
            }
        }
        __syncthreads();
        if (pending) {
            const double g1 = red[96], b1 = red[97], a1 = red[98];
            const bool conv = flag_set(red[99]), ok = flag_set(red[100]);
            if (conv) { result = 1; break; }
            if (it >= maxit) { result = 0; break; }
            // a step length the FP32 recurrences no longer give (p.Bh p from
            // them not positive): the inner solve has gone as far as FP32
            // takes it; the refinement continues from the iterate so far
            if (!ok) { result = 1; break; }
            gam = g1;
            beta = b1;
            alpha = a1;
            first = false;
        }
        const float af = (float)alpha, bf = (float)beta;
        const float *wc = m.w[cur];
        float *wn = m.w[cur ^ 1];
        float g = 0.f, dl = 0.f;
        int k = 0;
        for (int64_t i = R.first; i < n; i += R.step, ++k) {
            const float ri = S.get(0, k, i), ni = S.get(5, k, i);
            float wi;
            if constexpr (SM) wi = *S.vec(6, k);
            else wi = wc[i];
            float zi, si, pi;
            if (first) {
                zi = ni;
                si = wi;
                pi = ri;
            } else {
                zi = fmaf(bf, S.get(1, k, i), ni);
                si = fmaf(bf, S.get(2, k, i), wi);
                pi = fmaf(bf, S.get(3, k, i), ri);
            }
            const float di = fmaf(af, pi, S.get(4, k, i));
            const float rn = fmaf(-af, si, ri);
            const float wnx = fmaf(-af, zi, wi);
            S.put(1, k, i, zi);
            S.put(2, k, i, si);
            S.put(3, k, i, pi);
            S.put(4, k, i, di);
            S.put(0, k, i, rn);
            wn[i] = wnx;
            if constexpr (SM) {
                *S.vec(6, k) = wnx;
                m.d[i] = di;   // (stored, never read back: current at every grid barrier)
            }
            g = fmaf(rn, rn, g);
            dl = fmaf(wnx, rn, dl);
        }
        float sh[2] = {g, dl}, sl[2] = {0.f, 0.f};
        pend_slot = cur ? 7 : 4;
        if (!pipe_publish_pair<2>(sh, sl, pend_slot, m.a.part, red, m.a.ctrl)) return -2;
        ++it;
        cur ^= 1;
        pending = true;
    }
    return result;
}

// FP64 residual pass on the scaled system: rh = S b - Bh xh (own rows, into
// m.a.r), the sums ||b - B x||^2 and ||rh||^2.
__device__ bool pipe_mix_residual(const PipeMixArgs &m, int32_t n, double *red, double &rr, double &ss) {
    const PipeArgs &a = m.a;
    const Csr &cs = a.cs;
    const Rows R;
    double acc[2] = {0.0, 0.0};
    for (int64_t i = R.first; i < n; i += R.step) {
        const double si = a.sd[i];
        const double ri = a.b[i] * si - row_av(cs, a.ah, a.xh, n, i);
        a.r[i] = ri;
        const double ru = ri / si;
        acc[0] = fma(ru, ru, acc[0]);
        acc[1] = fma(ri, ri, acc[1]);
    }
    if (!pipe_publish<2>(acc, 0, a.part, red, a.ctrl)) return false;
    pipe_totals2(a, red, rr, ss);
    return true;
}

__global__ void __launch_bounds__(kPipeThreads, 1) pcgpipe_mix_kernel(PipeMixArgs m) {
    __shared__ double red[128];
    extern __shared__ __align__(16) double pipe_smem[];
    const PipeArgs &a = m.a;
    if (a.done && *a.done) return;
    const int32_t n = a.cs.n_dev ? *a.cs.n_dev : a.cs.n;
    const Csr &cs = a.cs;
    Ctrl *ctrl = a.ctrl;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const Rows R;
    // set-up (FP64): S, fl32(D), rh = S (b - B x), xh = S^-1 x; b.b, r.r
    double acc[2] = {0.0, 0.0};
    for (int64_t i = R.first; i < n; i += R.step) {
        double ri = a.b[i], d = 0.0;
        const int32_t e1 = cs.rp[i + 1];
        for (int32_t e = cs.rp[i]; e < e1; ++e) {
            const int32_t j = LC_IDX(cs.ci[e], n);
            const double v = cs.av[e];
            if (j == i) d = v;
            ri = fma(-v, ldcg(a.x + j), ri);
        }
        const double q = sqrt(d), si = 1.0 / q;
        a.sd[i] = si;
        a.d32[i] = (float)d;
        a.r[i] = si * ri;
        a.xh[i] = a.x[i] * q;
        acc[0] = fma(a.b[i], a.b[i], acc[0]);
        acc[1] = fma(ri, ri, acc[1]);
    }
    if (!pipe_publish<2>(acc, 0, a.part, red, ctrl)) return;
    double bb, rr;
    pipe_totals2(a, red, bb, rr);
    const double stop = (a.tol * a.tol) * bb;
    if (lead) {
        ctrl->bnorm2 = bb;
        ctrl->relres0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    if (bb == 0.0) {
        for (int64_t i = R.first; i < n; i += R.step) a.x[i] = 0.0;
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = 0.0; }
        return;
    }
    if (rr <= stop) {
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = sqrt(rr / bb); }
        return;
    }
    // Bh's values (FP64, FP32) of the own rows (S of the neighbours is
    // complete after the barrier), and ||rh||^2 of the set-up
    double ss0[1] = {0.0};
    for (int64_t i = R.first; i < n; i += R.step) {
        const double si = a.sd[i];
        const int32_t e1 = cs.rp[i + 1];
        for (int32_t e = cs.rp[i]; e < e1; ++e) {
            const int32_t j = LC_IDX(cs.ci[e], n);
            const double v = j == i ? 1.0 : cs.av[e] * si * ldcg(a.sd + j);
            a.ah[e] = v;
            m.ah32[e] = (float)v;
        }
        const double ri = a.r[i];
        ss0[0] = fma(ri, ri, ss0[0]);
    }
    if (!pipe_publish<1>(ss0, 2, a.part, red, ctrl)) return;
    double ss;
    {
        double t[1];
        if (threadIdx.x < 32) {
            pipe_totals<1>(2, a.part, t);
            if (threadIdx.x == 0) red[96] = t[0];
        }
        __syncthreads();
        ss = red[96];
        __syncthreads();
    }
    int it = 0, outer = 0, result = 0;
    float *smem32 = reinterpret_cast<float *>(pipe_smem);
    while (true) {
        if (rr <= stop) { result = 1; break; }
        if (outer >= m.max_outer || it >= a.maxit) { result = 0; break; }
        // the inner problem: r = fl32(rh / sigma), d = 0, w = fl32(Bh) r
        const double sigma = sqrt(ss), inv = 1.0 / sigma;
        for (int64_t i = R.first; i < n; i += R.step) m.r[i] = (float)(a.r[i] * inv);
        if (!grid_sync(ctrl, gridDim.x)) return;
        double acc2[2] = {0.0, 0.0};
        for (int64_t i = R.first; i < n; i += R.step) {
            const float wi = row_av32(cs, m.ah32, m.r, n, i), ri = m.r[i];
            m.w[0][i] = wi;
            m.d[i] = 0.f;
            acc2[0] = fma((double)ri, (double)ri, acc2[0]);
            acc2[1] = fma((double)wi, (double)ri, acc2[1]);
        }
        if (!pipe_publish<2>(acc2, 0, a.part, red, ctrl)) return;
        double g0, d0;
        pipe_totals2(a, red, g0, d0);
        // the inner target: inner_tol, or half of what the outer test still misses
        const double miss = sqrt(stop / rr);
        const double target = miss > m.inner_tol ? 0.5 * miss : m.inner_tol;
        const double istop = target * target * g0;
        const int r32 = n <= (int64_t)kPipeRowsSm * R.step
                            ? pipe_inner32<true>(m, n, red, smem32, g0, d0, istop, a.maxit, it)
                            : pipe_inner32<false>(m, n, red, smem32, g0, d0, istop, a.maxit, it);
        if (r32 == -2) return;
        if (r32 == -1) { result = -1; break; }
        // xh += sigma d (FP64), then the true residual
        for (int64_t i = R.first; i < n; i += R.step) a.xh[i] = fma(sigma, (double)m.d[i], a.xh[i]);
        if (!grid_sync(ctrl, gridDim.x)) return;
        if (!pipe_mix_residual(m, n, red, rr, ss)) return;
        ++outer;
    }
    for (int64_t i = R.first; i < n; i += R.step) a.x[i] = a.xh[i] * a.sd[i];
    if (lead) {
        ctrl->iters = it;
        ctrl->restarts = 0;
        ctrl->outer = outer;
        ctrl->converged = result;
        ctrl->early = 0;
        ctrl->relres = sqrt(rr / bb);
        if (result == -1) atomicCAS(&ctrl->status, LC_OK, LC_ERR_BREAKDOWN);
    }
}

}  // namespace

namespace {
int pipe_grid(const Csr &op, int grid_hint) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = sms;
    if (grid_hint > 0 && grid > grid_hint) grid = grid_hint;
    const int64_t units = ((int64_t)op.n + 32 * (kPipeWarps - 1) - 1) / (32 * (kPipeWarps - 1));
    if (grid > units) grid = units;
    if (grid > kMaxGrid) grid = kMaxGrid;
    return (int)(grid < 1 ? 1 : grid);
}

cudaError_t launch_pcg_csr_pipelined_mixed(const Csr &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                                           cudaStream_t s, bool after_cluster) {
    if (!after_cluster) {
        pipe_reset_kernel<<<1, 1, 0, s>>>(ctrl);
        note_launches(1);
    }
    PipeMixArgs m;
    PipeArgs &g = m.a;
    g.cs = op;
    g.b = a.b;
    g.x = a.x;
    g.ah = w.ahat;
    g.sd = w.dinv;
    g.d32 = w.r32;
    g.xh = w.xh;
    g.r = w.r;
    g.w[0] = w.q;
    g.w[1] = w.e0;
    g.z = w.z;
    g.s = w.p0;
    g.p = w.p1;
    g.n = w.e1;
    g.part = w.partials;
    g.tol = a.tol;
    g.maxit = a.maxit;
    g.max_restarts = a.max_restarts;
    g.ctrl = ctrl;
    g.done = after_cluster ? &ctrl->done : nullptr;
    // the FP32 inner vectors: the workspace's FP32 vectors, and two FP64
    // vectors the mixed solve does not otherwise use
    m.ah32 = w.val32;
    m.r = w.z32;
    m.w[0] = w.q32;
    m.w[1] = w.dinv32;
    m.z = w.p032;
    m.s = w.p132;
    m.p = w.x32;
    m.n = reinterpret_cast<float *>(w.e1);
    m.d = reinterpret_cast<float *>(w.z);
    m.inner_tol = a.inner_tol;
    m.max_outer = a.max_outer;
    const cudaError_t e = cudaFuncSetAttribute((const void *)pcgpipe_mix_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPipeSmBytes);
    if (e != cudaSuccess) return e;
    void *args[] = {&m};
    note_launches(1);
    return cudaLaunchCooperativeKernel((const void *)pcgpipe_mix_kernel, dim3((unsigned)pipe_grid(op, grid_hint)),
                                       dim3(kPipeThreads), args, kPipeSmBytes, s);
}
}  // namespace

cudaError_t launch_pcg_csr_pipelined(const Csr &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                                     cudaStream_t s, bool after_cluster) {
    if (a.precision == LC_PREC_MIXED) return launch_pcg_csr_pipelined_mixed(op, a, w, ctrl, grid_hint, s, after_cluster);
    if (!after_cluster) {
        pipe_reset_kernel<<<1, 1, 0, s>>>(ctrl);
        note_launches(1);
    }
    PipeArgs g;
    g.cs = op;
    g.b = a.b;
    g.x = a.x;
    g.ah = w.ahat;
    g.sd = w.dinv;
    g.d32 = w.r32;
    g.xh = w.xh;
    g.r = w.r;
    g.w[0] = w.q;
    g.w[1] = w.e0;
    g.z = w.z;
    g.s = w.p0;
    g.p = w.p1;
    g.n = w.e1;
    g.part = w.partials;
    g.tol = a.tol;
    g.maxit = a.maxit;
    g.max_restarts = a.max_restarts;
    g.ctrl = ctrl;
    g.done = after_cluster ? &ctrl->done : nullptr;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = sms;
    if (grid_hint > 0 && grid > grid_hint) grid = grid_hint;
    const int64_t units = ((int64_t)op.n + 32 * (kPipeWarps - 1) - 1) / (32 * (kPipeWarps - 1));
    if (grid > units) grid = units;
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (grid < 1) grid = 1;
    const cudaError_t e = cudaFuncSetAttribute((const void *)pcgpipe_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPipeSmBytes);
    if (e != cudaSuccess) return e;
    void *args[] = {&g};
    note_launches(1);
    return cudaLaunchCooperativeKernel((const void *)pcgpipe_kernel, dim3((unsigned)grid), dim3(kPipeThreads), args,
                                       kPipeSmBytes, s);
}

}  // namespace lc
