// lc_pcg1.cu -- Jacobi-PCG with ONE grid-wide reduction per iteration
// (the Chronopoulos-Gear arrangement) for CSR systems whose solve is bound by
// barrier latency: the extracted local subsystem of Alg 1 (step 5).
//
// It produces the iterates of the two-reduction form in exact arithmetic
// (the same x_i, r_i, p_i, alpha_i, beta_i), arranged so that the two dot
// products of an iteration are taken together.  With M = diag(A)^-1,
// u = M r and w = A u:
//   s_i = A p_i is carried by recurrence, s_i = w_i + beta_i s_(i-1)
//   gamma_i = (r_i, u_i),  delta_i = (w_i, u_i)
//   beta_i = gamma_i / gamma_(i-1),  alpha_i = gamma_i / (delta_i - beta_i gamma_i / alpha_(i-1))
// One grid-wide phase per iteration, for every own row i:
//   u_i = dinv_i r_i;  p_i = u_i + beta p_i;  s_i = w_i + beta s_i;  x_i += alpha p_i
//   r'_i = r_i - alpha s_i;  u'_i = dinv_i r'_i
//   w'_i = sum_j a_ij u'_j, every neighbour's u'_j recomputed from its r_j,
//          s_j, w_j of this iteration -- so no barrier separates the vector
//          updates from the product
//   partials (r', u'), (w', u'), (r', r')
// then one grid reduction (which is also the iteration's only barrier); thread
// 0 of each block derives beta', alpha' and the stopping and breakdown flags.
// r, s and w are double-buffered: neighbours read this iteration's copy while
// the owner writes the next one; p and x are touched by their owner only.
// Stopping test, true-residual confirmation and restarts are those of the
// two-reduction kernel (lc_pcg_impl.cuh), with the same Ctrl fields.
#include "lc_internal.cuh"

namespace lc {

namespace {

constexpr int kThreads = 256;

struct Cg1Args {
    Csr cs;
    const double *b;
    double *x;
    double *r[2], *s[2], *w[2];
    double *p;
    const double *dinv;
    double *part;
    double tol;
    int maxit, max_restarts;
    Ctrl *ctrl;
    const int32_t *done;   // set: a cluster kernel launched before may already have solved it
};

__global__ void csr_dinv1_kernel(Csr c, double *dinv) {
    const int32_t n = c.n_dev ? *c.n_dev : c.n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        const int32_t e1 = c.rp[i + 1];
        for (int32_t e = c.rp[i]; e < e1; ++e)
            if (c.ci[e] == i) d = c.av[e];
        dinv[i] = 1.0 / d;
    }
}

__global__ void reset1_kernel(Ctrl *ctrl) {
    ctrl->bar_count = 0;
    ctrl->iters = 0;
    ctrl->restarts = 0;
    ctrl->outer = 0;
    ctrl->converged = 0;
    ctrl->early = 0;
}

// r = b - A x into r[0] (own rows), then w = A u (u = dinv r, neighbours'
// recomputed from their r) into w[0]; returns the sums b.b, r.r, gamma,
// delta.  Two grid barriers.
__device__ bool cg1_setup(const Cg1Args &a, int32_t n, double *red, double &bb, double &rr, double &gam,
                          double &del) {
    const Csr &cs = a.cs;
    double acc[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        double ri = a.b[i];
        const int32_t e1 = cs.rp[i + 1];
        for (int32_t e = cs.rp[i]; e < e1; ++e) ri = fma(-cs.av[e], ldcg(a.x + LC_IDX(cs.ci[e], n)), ri);
        a.r[0][i] = ri;
        acc[0] = fma(a.b[i], a.b[i], acc[0]);
        acc[1] = fma(ri, ri, acc[1]);
    }
    double o[2];
    if (!grid_sums<2, 0, double>(acc, 0, a.part, red, a.ctrl, o)) return false;
    bb = o[0];
    rr = o[1];
    double acc2[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        double wi = 0.0;
        const int32_t e1 = cs.rp[i + 1];
        for (int32_t e = cs.rp[i]; e < e1; ++e) {
            const int32_t j = LC_IDX(cs.ci[e], n);
            wi = fma(cs.av[e], a.dinv[j] * ldcg(a.r[0] + j), wi);
        }
        const double ri = a.r[0][i], ui = a.dinv[i] * ri;
        a.w[0][i] = wi;
        acc2[0] = fma(ri, ui, acc2[0]);
        acc2[1] = fma(wi, ui, acc2[1]);
    }
    double o2[2];
    if (!grid_sums<2, 0, double>(acc2, 2, a.part, red, a.ctrl, o2)) return false;
    gam = o2[0];
    del = o2[1];
    return true;
}

// Iterations from the state cg1_setup left (r[0], w[0], gamma, delta); x is
// updated in place, so a restart only needs cg1_setup again.  Returns 1
// converged, 0 iteration limit, -1 breakdown, -2 wait timed out.
__device__ int cg1_iterations(const Cg1Args &a, int32_t n, double *red, double gam, double del, double stop,
                              int &it) {
    const Csr &cs = a.cs;
    if (!(del > 0.0) || !isfinite(del)) return -1;
    double alpha = gam / del, beta = 0.0;
    bool first = true;
    int cur = 0;
    while (true) {
        const double *rc = a.r[cur], *sc = a.s[cur], *wc = a.w[cur];
        double *rn = a.r[cur ^ 1], *sn = a.s[cur ^ 1], *wn = a.w[cur ^ 1];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
            const double di = a.dinv[i], ri = ldcg(rc + i);
            const double ui = di * ri;
            const double pi = first ? ui : fma(beta, a.p[i], ui);
            const double si = first ? ldcg(wc + i) : fma(beta, ldcg(sc + i), ldcg(wc + i));
            a.x[i] = fma(alpha, pi, a.x[i]);
            const double rn_i = fma(-alpha, si, ri);
            const double un_i = di * rn_i;
            double wi = 0.0;
            const int32_t e1 = cs.rp[i + 1];
            for (int32_t e = cs.rp[i]; e < e1; ++e) {
                const int32_t j = LC_IDX(cs.ci[e], n);
                double uj;
                if (j == i) {
                    uj = un_i;
                } else {
                    const double sj = first ? ldcg(wc + j) : fma(beta, ldcg(sc + j), ldcg(wc + j));
                    uj = a.dinv[j] * fma(-alpha, sj, ldcg(rc + j));
                }
                wi = fma(cs.av[e], uj, wi);
            }
            a.p[i] = pi;
            sn[i] = si;
            rn[i] = rn_i;
            wn[i] = wi;
            acc[0] = fma(rn_i, un_i, acc[0]);
            acc[1] = fma(wi, un_i, acc[1]);
            acc[2] = fma(rn_i, rn_i, acc[2]);
        }
        double o[6];   // gamma', delta', r'.r', converged, beta', alpha' (0 on breakdown)
        const double g0 = gam, a0 = alpha;
        // alternate slot sets: a block may already write the next iteration's
        // partials while a slower one still reads these
        if (!grid_sums<3, 3, double>(acc, cur ? 7 : 4, a.part, red, a.ctrl, o, [g0, a0, stop](double *t) {
                t[3] = t[2] <= stop ? 1.0 : 0.0;
                const double bt = t[0] / g0;
                const double den = t[1] - bt * t[0] / a0;
                const bool ok = den > 0.0 && isfinite(den);
                t[4] = bt;
                t[5] = ok ? t[0] / den : 0.0;
            }))
            return -2;
        ++it;
        cur ^= 1;
        if (flag_set(o[3])) return 1;
        if (it >= a.maxit) return 0;
        if (!flag_set(o[5])) return -1;
        gam = o[0];
        beta = o[4];
        alpha = o[5];
        first = false;
    }
}

__global__ void __launch_bounds__(kThreads, 3) pcg1_kernel(Cg1Args a) {
    __shared__ double red[128];
    if (a.done && *a.done) return;
    const int32_t n = a.cs.n_dev ? *a.cs.n_dev : a.cs.n;
    Ctrl *ctrl = a.ctrl;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    double bb, rr, gam, del;
    if (!cg1_setup(a, n, red, bb, rr, gam, del)) return;
    const double stop = (a.tol * a.tol) * bb;
    if (lead) {
        ctrl->bnorm2 = bb;
        ctrl->relres0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    if (bb == 0.0) {
        for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
            a.x[i] = 0.0;
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = 0.0; }
        return;
    }
    if (rr <= stop) {
        if (lead) { ctrl->converged = 1; ctrl->early = 1; ctrl->relres = sqrt(rr / bb); }
        return;
    }
    int it = 0, restarts = 0, result;
    while (true) {
        result = cg1_iterations(a, n, red, gam, del, stop, it);
        if (result == -2) return;
        if (result != 1) break;
        // converged on the recurrence residual: confirm with the true one
        double bb2;
        if (!cg1_setup(a, n, red, bb2, rr, gam, del)) return;
        if (rr <= stop) break;
        result = 0;
        if (++restarts > a.max_restarts || it >= a.maxit) break;
    }
    if (result == 0 && it >= a.maxit) {   // report the true residual of the last iterate
        double bb2, g2, d2;
        if (!cg1_setup(a, n, red, bb2, rr, g2, d2)) return;
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

}  // namespace

cudaError_t launch_pcg_csr_single(const Csr &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                                  cudaStream_t s, bool after_cluster) {
    csr_dinv1_kernel<<<152 * 4, 256, 0, s>>>(op, w.dinv);
    note_launches(1);
    if (!after_cluster) {
        reset1_kernel<<<1, 1, 0, s>>>(ctrl);
        note_launches(1);
    }
    Cg1Args g;
    g.cs = op;
    g.b = a.b;
    g.x = a.x;
    g.r[0] = w.r; g.r[1] = w.z;
    g.s[0] = w.p0; g.s[1] = w.p1;
    g.w[0] = w.q; g.w[1] = w.e0;
    g.p = w.e1;
    g.dinv = w.dinv;
    g.part = w.partials;
    g.tol = a.tol;
    g.maxit = a.maxit;
    g.max_restarts = a.max_restarts;
    g.ctrl = ctrl;
    g.done = after_cluster ? &ctrl->done : nullptr;
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg1_kernel, kThreads, 0);
    int64_t grid = (int64_t)sms * (per < 1 ? 1 : per);
    if (grid_hint > 0 && grid > grid_hint) grid = grid_hint;
    const int64_t units = ((int64_t)op.n + kThreads - 1) / kThreads;
    if (grid > units) grid = units;
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (grid < 1) grid = 1;
    void *args[] = {&g};
    note_launches(1);
    return cudaLaunchCooperativeKernel((const void *)pcg1_kernel, dim3((unsigned)grid), dim3(kThreads), args, 0, s);
}

}  // namespace lc
