// lc_cluster.cu -- the local subsystem solve (Alg 1, step 5: Jacobi-PCG on
// the extracted system B xL = rhs) on ONE thread-block cluster.
//
// The local system is small (K of a few 10^4 rows for a percent-sized
// domain), so a grid-wide solve spends its time in grid barriers, not in
// arithmetic.  Here one cluster of C CTAs (16 where the GPU schedules it,
// else 8 or 4) keeps every vector of the solve in distributed shared memory:
// CTA c owns rows [c R, (c+1) R), R = ceil(K / C), and holds x, r, z, q,
// dinv and two buffers of p of those rows.  A row's neighbours are read from
// the owning CTA's shared memory (DSMEM) and the cluster synchronises with
// its hardware barrier.  The matrix itself is read from global memory (L2
// resident after the first iteration).
//
// Per iteration, two cluster barriers (hardware barriers, cheap next to a
// grid-wide one):
//   phase A  q_i = sum_j a_ij p_j with p_j = z_j + beta p_old,j formed from
//            the owner's z and previous p; p_i stored into the other buffer;
//            block partial p.q  (barrier: every CTA has stored its partial
//            in every CTA's slot row)
//   phase B  alpha = rz / pq; x += alpha p; r -= alpha q; z = dinv r;
//            partials r.z and r.r                          (barrier)
// Each CTA adds the C slot rows by the same shuffle tree, so every CTA takes
// the same decisions.  Iteration, stopping test, true-residual confirmation
// and restarts follow the grid kernel of lc_pcg_impl.cuh (same Ctrl
// fields).
//
// The kernel first decides whether to take the system (K <= max_rows and the
// rows fit); it records the decision in ctrl->done, and the grid kernel
// launched after it returns at once when the cluster already solved the
// system.
#include "lc_pcg_impl.cuh"   // FP32-pair helpers (split_f2, f2_add_prod)

#include <cooperative_groups.h>

#include <mutex>

namespace cg = cooperative_groups;

namespace lc {

namespace {

constexpr int kClThreads = 1024;
constexpr int kClMax = 16;
constexpr int kClVecs = 7;                                  // x, r, z, q, dinv, p, p (previous)
constexpr int kClUnroll = 5;                                // row entries loaded together
constexpr int kClFixed = (3 * kClMax * 4 + 128) * 8;        // three slot arrays + block-sum scratch

struct ClMem {
    double *slotS, *slotA, *slotB;   // [kClMax][4]: partial sums, one row per source CTA
    double *red;                     // block_sum scratch (128)
    double *x, *r, *z, *q, *dinv, *p, *p2;
};

__device__ __forceinline__ ClMem carve_cl(double *base, int rcap) {
    ClMem m;
    m.slotS = base;
    m.slotA = base + kClMax * 4;
    m.slotB = base + 2 * kClMax * 4;
    m.red = base + 3 * kClMax * 4;
    double *v = m.red + 128;
    const size_t rc = (size_t)rcap;
    m.x = v;
    m.r = v + rc;
    m.z = v + 2 * rc;
    m.q = v + 3 * rc;
    m.dinv = v + 4 * rc;
    m.p = v + 5 * rc;
    m.p2 = v + 6 * rc;
    return m;
}

struct ClNoPost {
    __device__ void operator()(double *) const {}
};

// Cluster-wide sums of NV per-thread values: block sum, the block's result
// stored into slot row `rank` of every CTA, cluster barrier, and warp 0 of
// each CTA adds the C rows by a fixed shuffle tree (identical results in
// every CTA; log2 C dependent FP64 additions instead of C -- an FP64 warp
// instruction holds the FP64 pipe as long with one active lane as with 32);
// thread 0 runs post(t) on the totals, which may append ND derived scalars
// (the step lengths; one FP64 division per CTA instead of one per thread).
// Every thread reads totals and derived values back from shared memory.
template <int NV, int ND = 0, class Post = ClNoPost>
__device__ __forceinline__ void cl_sums(cg::cluster_group &cl, double (&v)[NV], double *slots, double *red, int C,
                                        double (&out)[NV + ND], Post post = Post()) {
    block_sum<NV, double>(v, red);   // lane 0 of warp 0 holds the block sums
    const int rank = (int)cl.block_rank();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = __shfl_sync(kFull, v[k], 0);
        if ((int)threadIdx.x < C) {
            double *dst = cl.map_shared_rank(slots, (unsigned)threadIdx.x);
#pragma unroll
            for (int k = 0; k < NV; ++k) dst[rank * 4 + k] = v[k];
        }
    }
    cl.sync();
    if (threadIdx.x < 32) {
        const int lane = (int)threadIdx.x;
        int top = 1;
        while (top < C) top <<= 1;
        double t[NV + ND];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < C ? slots[lane * 4 + k] : 0.0;
            for (int o = top >> 1; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
            t[k] = s;
        }
        if (lane == 0) {
            post(t);
#pragma unroll
            for (int k = 0; k < NV + ND; ++k) red[96 + k] = t[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV + ND; ++k) out[k] = red[96 + k];
}

// cl_sums on FP32 pairs: value k of a thread is (h[k] + l[k]) 2^e[k]; the
// warps, the block and the cluster add pairs with FP32 two-sums, and only the
// totals become FP64 (each block sum's FP64 shuffle tree cost about as much
// FP64 issue as the rows' own arithmetic).  The slot rows hold the blocks'
// pairs.
template <int NV, int ND = 0, class Post = ClNoPost>
__device__ __forceinline__ void cl_sums_pair(cg::cluster_group &cl, float (&h)[NV], float (&l)[NV],
                                             const int (&e)[NV], double *slots, double *red, int C,
                                             double (&out)[NV + ND], Post post = Post()) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float bh = __shfl_down_sync(kFull, h[k], o), bl = __shfl_down_sync(kFull, l[k], o);
            pair_add(h[k], l[k], bh, bl);
        }
    float *fs = reinterpret_cast<float *>(red);   // 2 NV x 32 floats
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) { fs[(2 * k) * 32 + warp] = h[k]; fs[(2 * k + 1) * 32 + warp] = l[k]; }
    __syncthreads();
    const int rank = (int)cl.block_rank();
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
                const float bh = __shfl_sync(kFull, h[k], lane + o), bl = __shfl_sync(kFull, l[k], lane + o);
                if (lane + o < 32) pair_add(h[k], l[k], bh, bl);
            }
#pragma unroll
        for (int k = 0; k < NV; ++k) { h[k] = __shfl_sync(kFull, h[k], 0); l[k] = __shfl_sync(kFull, l[k], 0); }
        if (lane < C) {
            float2 *dst = reinterpret_cast<float2 *>(cl.map_shared_rank(slots, (unsigned)lane));
#pragma unroll
            for (int k = 0; k < NV; ++k) dst[rank * 4 + k] = make_float2(h[k], l[k]);
        }
    }
    cl.sync();
    if (warp == 0) {
        int top = 1;
        while (top < C) top <<= 1;
        const float2 *src = reinterpret_cast<const float2 *>(slots);
        double t[NV + ND];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            float sh = 0.f, sl = 0.f;
            if (lane < C) { const float2 v = src[lane * 4 + k]; sh = v.x; sl = v.y; }
            for (int o = top >> 1; o > 0; o >>= 1) {
                const float bh = __shfl_down_sync(kFull, sh, o), bl = __shfl_down_sync(kFull, sl, o);
                pair_add(sh, sl, bh, bl);
            }
            t[k] = ldexp((double)sh + (double)sl, e[k]);
        }
        if (lane == 0) {
            post(t);
#pragma unroll
            for (int k = 0; k < NV + ND; ++k) red[96 + k] = t[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV + ND; ++k) out[k] = red[96 + k];
}

__device__ __forceinline__ bool cl_flag(double f) { return __double_as_longlong(f) != 0; }

// Row partition: owner of row j = j / R, computed in FP32 (exact for
// j < 2^24, which every system the cluster takes satisfies) and corrected.
struct ClPart {
    int R;
    float inv;
    int K;   // rows of the system (the range of a column index)
    __device__ __forceinline__ int owner(int j) const {
        int o = (int)((float)j * inv);
        if (o * R > j) --o;
        else if ((o + 1) * R <= j) ++o;
        return o;
    }
};

// Row j's entry of a distributed vector (`vec` = this CTA's array; the same
// offset in the owner's shared memory).
__device__ __forceinline__ double cl_load(cg::cluster_group &cl, double *vec, int j, const ClPart &pt, int rank) {
    j = LC_IDX(j, pt.K);
    const int owner = pt.owner(j);
    const int lj = j - owner * pt.R;
    if (owner == rank) return vec[lj];
    return cl.map_shared_rank(vec, (unsigned)owner)[lj];
}

// sum_e a_e v_(col e) over the row's entries in ascending order; the first
// kClUnroll entries are loaded together.
__device__ __forceinline__ double cl_row_dot(cg::cluster_group &cl, const Csr &cs, int i, double *vec,
                                            const ClPart &pt, int rank) {
    const int e0 = cs.rp[i], e1 = cs.rp[i + 1];
    int jj[kClUnroll];
    double aa[kClUnroll];
#pragma unroll
    for (int t = 0; t < kClUnroll; ++t) {
        const bool in = e0 + t < e1;
        jj[t] = in ? __ldg(cs.ci + e0 + t) : -1;
        aa[t] = in ? __ldg(cs.av + e0 + t) : 0.0;
    }
    double vv[kClUnroll];
#pragma unroll
    for (int t = 0; t < kClUnroll; ++t) vv[t] = jj[t] >= 0 ? cl_load(cl, vec, jj[t], pt, rank) : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < kClUnroll; ++t)
        if (jj[t] >= 0) acc = fma(aa[t], vv[t], acc);
    for (int e = e0 + kClUnroll; e < e1; ++e) acc = fma(__ldg(cs.av + e), cl_load(cl, vec, __ldg(cs.ci + e), pt, rank), acc);
    return acc;
}

// q_i = sum_e a_e p_(col e) with p_j = z_j + beta p_old,j (p_j = z_j on the
// first iteration) formed where it is read, from the owners' z and p_old;
// *pi receives p_i.  The same value of p_j as its owner forms for itself.
__device__ __forceinline__ double cl_row_dot_p(cg::cluster_group &cl, const Csr &cs, int i, double *z, double *pold,
                                              bool first, double beta, const ClPart &pt, int rank, double *pi) {
    const int e0 = cs.rp[i], e1 = cs.rp[i + 1];
    double acc = 0.0, pc = 0.0;
    const auto pat = [&](int j) {
        const double zj = cl_load(cl, z, j, pt, rank);
        return first ? zj : fma(beta, cl_load(cl, pold, j, pt, rank), zj);
    };
    int jj[kClUnroll];
    double aa[kClUnroll];
#pragma unroll
    for (int t = 0; t < kClUnroll; ++t) {
        const bool in = e0 + t < e1;
        jj[t] = in ? __ldg(cs.ci + e0 + t) : -1;
        aa[t] = in ? __ldg(cs.av + e0 + t) : 0.0;
    }
    double vv[kClUnroll];
#pragma unroll
    for (int t = 0; t < kClUnroll; ++t) vv[t] = jj[t] >= 0 ? pat(jj[t]) : 0.0;
#pragma unroll
    for (int t = 0; t < kClUnroll; ++t)
        if (jj[t] >= 0) {
            if (jj[t] == i) pc = vv[t];
            acc = fma(aa[t], vv[t], acc);
        }
    for (int e = e0 + kClUnroll; e < e1; ++e) {
        const int j = __ldg(cs.ci + e);
        const double pj = pat(j);
        if (j == i) pc = pj;
        acc = fma(__ldg(cs.av + e), pj, acc);
    }
    *pi = pc;
    return acc;
}

__global__ void __launch_bounds__(kClThreads, 1)
    cluster_pcg_kernel(Csr cs, const double *__restrict__ b, double *xg, double tol, int maxit, int max_restarts,
                       int rcap, int max_rows, Ctrl *ctrl) {
    extern __shared__ __align__(16) double cl_smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int K = cs.n_dev ? *cs.n_dev : cs.n;
    const bool lead = rank == 0 && threadIdx.x == 0;
    const int R = K > 0 ? (K + C - 1) / C : 1;
    if (R > rcap || K > max_rows) {   // not taken: hand over to the grid kernel, with the state it expects
        if (lead) {
            ctrl->done = 0;
            ctrl->bar_count = 0;
            ctrl->iters = 0;
            ctrl->restarts = 0;
            ctrl->outer = 0;
            ctrl->converged = 0;
            ctrl->early = 0;
        }
        return;
    }
    if (lead) {
        ctrl->done = 1;
        ctrl->iters = 0;
        ctrl->restarts = 0;
        ctrl->outer = 0;
        ctrl->converged = 0;
        ctrl->early = 0;
    }
    const ClMem m = carve_cl(cl_smem, rcap);
    const ClPart pt{R, 1.0f / (float)R, K};
    const int r0 = min(K, rank * R), r1 = min(K, r0 + R);
    const int tid = (int)threadIdx.x, nth = (int)blockDim.x;

    for (int i = r0 + tid; i < r1; i += nth) {
        const int li = i - r0;
        m.x[li] = xg[i];
        double d = 0.0;
        const int e1 = cs.rp[i + 1];
        for (int e = cs.rp[i]; e < e1; ++e)
            if (cs.ci[e] == i) d = cs.av[e];
        m.dinv[li] = 1.0 / d;
    }
    cl.sync();   // every x in place before any row reads its neighbours

    // r = b - B x, z = dinv r; cluster sums of b.b, r.z, r.r
    auto residual = [&](double &bb, double &rz, double &rr) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int i = r0 + tid; i < r1; i += nth) {
            const int li = i - r0;
            const double ax = cl_row_dot(cl, cs, i, m.x, pt, rank);
            const double bi = b[i];
            const double ri = bi - ax;
            const double zi = m.dinv[li] * ri;
            m.r[li] = ri;
            m.z[li] = zi;
            acc[0] = fma(bi, bi, acc[0]);
            acc[1] = fma(ri, zi, acc[1]);
            acc[2] = fma(ri, ri, acc[2]);
        }
        double out[3];
        cl_sums<3>(cl, acc, m.slotS, m.red, C, out);
        bb = out[0];
        rz = out[1];
        rr = out[2];
    };

    // CG iterations from the current r, z; 1 converged (recurrence residual),
    // 0 iteration limit, -1 breakdown
    // p is formed inside the product from z and the previous p (two buffers,
    // swapped every iteration), so no barrier separates its update from the
    // product: two cluster barriers per iteration
    double *pbuf[2] = {m.p, m.p2};
    auto iterate = [&](double rz, double stop, int &it) -> int {
        bool first = true;
        double beta = 0.0;
        int cur = 0;
        double rr_last = rz;   // the scale of the stopping norm's pairs
        while (true) {
            double *p = pbuf[cur], *pold = pbuf[cur ^ 1];
            // the sums on FP32 pairs of the values scaled by 2^-ps, ps half the
            // exponent of r.z (r.r: of its last total)
            const int ps = ((int)((__double_as_longlong(rz) >> 52) & 0x7ff) - 1023) >> 1;
            const int pr = ((int)((__double_as_longlong(rr_last) >> 52) & 0x7ff) - 1023) >> 1;
            float h1[1] = {0.f}, l1[1] = {0.f};
            for (int i = r0 + tid; i < r1; i += nth) {
                const int li = i - r0;
                double pi;
                const double qi = cl_row_dot_p(cl, cs, i, m.z, pold, first, beta, pt, rank, &pi);
                p[li] = pi;
                m.q[li] = qi;
                float ph, pl, qh, ql;
                split_f2(pi, ps, ph, pl);
                split_f2(qi, ps, qh, ql);
                f2_add_prod(ph, pl, qh, ql, h1[0], l1[0]);
            }
            double o1[3];   // p.q, alpha, breakdown flag
            const int e1[1] = {2 * ps};
            cl_sums_pair<1, 2>(cl, h1, l1, e1, m.slotA, m.red, C, o1, [rz](double *t) {
                const bool ok = t[0] > 0.0 && isfinite(t[0]);
                t[1] = ok ? rz / t[0] : 0.0;
                t[2] = ok ? 0.0 : 1.0;
            });
            if (cl_flag(o1[2])) return -1;
            const double alpha = o1[1];
            float h2[2] = {0.f, 0.f}, l2[2] = {0.f, 0.f};
            for (int i = r0 + tid; i < r1; i += nth) {
                const int li = i - r0;
                const double xi = fma(alpha, p[li], m.x[li]);
                const double ri = fma(-alpha, m.q[li], m.r[li]);
                const double zi = m.dinv[li] * ri;
                m.x[li] = xi;
                m.r[li] = ri;
                m.z[li] = zi;
                float rh, rl, zh, zl, sh, sl;
                split_f2(ri, ps, rh, rl);
                split_f2(zi, ps, zh, zl);
                split_f2(ri, pr, sh, sl);
                f2_add_prod(rh, rl, zh, zl, h2[0], l2[0]);
                f2_add_prod(sh, sl, sh, sl, h2[1], l2[1]);
            }
            double o2[4];   // r.z, r.r, converged flag, beta
            const int e2[2] = {2 * ps, 2 * pr};
            cl_sums_pair<2, 2>(cl, h2, l2, e2, m.slotB, m.red, C, o2, [rz, stop](double *t) {
                t[2] = t[1] <= stop ? 1.0 : 0.0;
                t[3] = t[0] / rz;
            });
            ++it;
            if (cl_flag(o2[2])) return 1;
            if (it >= maxit) return 0;
            beta = o2[3];
            rz = o2[0];
            rr_last = o2[1];
            first = false;
            cur ^= 1;
        }
    };

    double bb, rz, rr;
    residual(bb, rz, rr);
    const double stop = (tol * tol) * bb;
    if (lead) {
        ctrl->bnorm2 = bb;
        ctrl->relres0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    if (bb == 0.0) {   // B x = 0: x = 0
        for (int i = r0 + tid; i < r1; i += nth) xg[i] = 0.0;
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = 0.0; }
        cl.sync();
        return;
    }
    if (rr <= stop) {   // the starting iterate is returned as it is
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = sqrt(rr / bb); }
        cl.sync();
        return;
    }
    int it = 0, restarts = 0, result;
    while (true) {
        result = iterate(rz, stop, it);
        if (result != 1) break;
        double bb2;   // converged on the recurrence residual: confirm with the true one
        residual(bb2, rz, rr);
        if (rr <= stop) break;
        result = 0;
        if (++restarts > max_restarts || it >= maxit) break;
    }
    if (result == 0 && it >= maxit) {   // report the true residual of the last iterate
        double bb2, rz2;
        residual(bb2, rz2, rr);
    }
    for (int i = r0 + tid; i < r1; i += nth) xg[i] = m.x[i - r0];
    if (lead) {
        ctrl->iters = it;
        ctrl->restarts = restarts;
        ctrl->converged = result;
        ctrl->early = 0;
        ctrl->relres = sqrt(rr / bb);
        if (result == -1) atomicCAS(&ctrl->status, LC_OK, LC_ERR_BREAKDOWN);
    }
    cl.sync();   // no CTA leaves while another may still address its shared memory
}

struct ClConfig {
    int C = 0;          // cluster size, 0 = not available
    int rcap = 0;       // rows per CTA
    size_t smem = 0;    // dynamic shared memory per CTA
};

ClConfig probe_cluster(int dev) {
    ClConfig c;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return c;
    const size_t smem = (size_t)optin;
    if (smem <= (size_t)kClFixed + kClVecs * 8 * 1024) return c;
    const void *k = (const void *)cluster_pcg_kernel;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return c;
    }
    for (int C : {16, 8, 4}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(kClThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, cluster_pcg_kernel, &cfg) == cudaSuccess && n >= 1) {
            c.C = C;
            c.smem = smem;
            c.rcap = (int)((smem - kClFixed) / (kClVecs * sizeof(double)));
            return c;
        }
        cudaGetLastError();
    }
    return c;
}

ClConfig cluster_config() {
    static std::mutex mu;
    static ClConfig cfg[64];
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return ClConfig{};
    std::lock_guard<std::mutex> g(mu);
    if (!done[dev]) {
        cfg[dev] = probe_cluster(dev);
        done[dev] = true;
    }
    return cfg[dev];
}

}  // namespace

int cluster_local_rows() {
    const ClConfig c = cluster_config();
    return c.C * c.rcap;
}

cudaError_t launch_pcg_csr_cluster(const Csr &op, const PcgArgs &a, int max_rows, int threads, int ctas, Ctrl *ctrl,
                                   cudaStream_t s) {
    const ClConfig c = cluster_config();
    if (c.C == 0) return cudaErrorNotSupported;
    if (threads < 32 || threads > kClThreads || threads % 32) return cudaErrorInvalidValue;
    // fewer CTAs than the largest cluster the GPU schedules: cheaper barriers,
    // less FP64 throughput (the kernel hands larger systems to the grid kernel)
    const int C = ctas > 0 && ctas < c.C ? ctas : c.C;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    note_launches(1);
    return cudaLaunchKernelEx(&cfg, cluster_pcg_kernel, op, a.b, a.x, a.tol, (int)a.maxit, (int)a.max_restarts,
                              c.rcap, max_rows, ctrl);
}

}  // namespace lc
