// lc_api.cu -- host implementation of the C ABI declared in include/lc_api.h.
//
// Argument checking, workspace ownership and the stream-ordered sequencing
// of the kernels of lc_mark.cu, lc_extract.cu and lc_pcg*.cu.  No entry point
// of the hot path allocates, synchronises or copies to the host unless it
// is asked for host statistics.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <atomic>
#include <mutex>

#include "lc_internal.cuh"

namespace lc {
static std::atomic<long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// the check words of the translation units of a bounds-checked build
static std::mutex g_check_mu;
static std::vector<std::pair<unsigned (*)(), const char *>> &check_units() {
    static std::vector<std::pair<unsigned (*)(), const char *>> v;
    return v;
}
void register_check_word(unsigned (*take)(), const char *unit) {
    std::lock_guard<std::mutex> g(g_check_mu);
    check_units().push_back({take, unit});
}
#ifdef LC_CHECKED
namespace {
__device__ int g_selftest_probe[4];
__global__ void checked_selftest_kernel(int i) { g_selftest_probe[LC_IDX(i, 4)] += 1; }
}  // namespace
#endif
}  // namespace lc

struct lc_ctx {
    int device = 0;
    int sms = 0;
    std::string err;
    // one reference held by the caller (released by lc_ctx_destroy) and one
    // per operator or batch created on the context: whichever release comes
    // last frees it, so the destruction order does not matter
    std::atomic<int> refs{1};
};

namespace {
void ctx_ref(lc_ctx *c) { c->refs.fetch_add(1, std::memory_order_relaxed); }
void ctx_unref(lc_ctx *c) {
    if (c && c->refs.fetch_sub(1, std::memory_order_acq_rel) == 1) delete c;
}
}  // namespace

struct lc_op {
    lc_ctx *ctx = nullptr;
    int kind = 0;   // 0 stencil, 1 csr
    lc::Stencil st{};
    lc::Csr csr{};
    int64_t n = 0, nnz = 0;
    // owned device memory
    void *arena = nullptr;
    lc::Ctrl *ctrl = nullptr;        // marking / global solve
    lc::Ctrl *ctrl_loc = nullptr;    // local solve
    double *dinv = nullptr;
    float *D32 = nullptr, *Tx32 = nullptr, *Ty32 = nullptr, *Tz32 = nullptr, *dinv32 = nullptr;
    double *work = nullptr;          // residual / gradient (N)
    uint8_t *mask_tmp = nullptr, *mask_own = nullptr;
    uint32_t *bits_a = nullptr, *bits_b = nullptr;   // stencils: bit-packed mask rows (threshold, dilation)
    double *tree_a = nullptr, *tree_b = nullptr;
    lc::ExtractWork ew{};
    lc_subsys sub{};                 // internal subsystem buffers
    lc::PcgWork pw{};
    cudaEvent_t ev[8] = {};
    // tuning knobs (lc_op_set_tuning)
    int pcg_minblocks = 3;   // register budget of the structured-grid PCG kernel
    int pcg_grid_cap = 0;    // blocks of the global PCG launch (0: as many as fit)
    const uint8_t *colour = nullptr;    // CSR: caller's colouring for Gauss-Seidel (device)
    int ncolours = 0;
    // local solves of up to this many rows on one thread-block cluster of
    // 256-thread CTAs: measured faster than the grid kernel below ~8K rows
    int local_cluster_rows = 2048;
    int local_single = 0;               // local solves: one grid reduction per iteration
    int local_pipelined = 1;            // local solves: pipelined CG, one grid barrier per iteration
    int local_grid_cap = 0;             // local solves: blocks of the grid kernel (0 = one per SM)
    int local_cluster_threads = 256;
    int local_cluster_ctas = 0;         // CTAs of that cluster (0: the largest the GPU schedules)
    int pcg_scaled = 1;      // 2D FP64: iterate on D^-1/2 A D^-1/2 (fewer FP64 instructions)
    int pcg_big = 1;         // 2D solves: one 768-thread block per SM (2 % faster at 2048^2, mixed 5 %)
    int pcg_pairdot = 1;     // 2D scaled wide FP64: dots and block sums on FP32 pairs (7 % faster at 2048^2)
    int pcg_lazy_x = 1;      // 2D scaled wide FP64 pair: x update in the next phase A (4.6 % faster at 2048^2)
    int csr_store_p = 1;     // global CSR solves: p stored once per row before the product
    int pcg_wide = 1;        // 2D scaled FP64: four cells per lane (when nx % 4 == 0; 3.5 % faster at 2048^2)
    double *sc = nullptr, *sq = nullptr, *Txh = nullptr, *Tyh = nullptr, *Tzh = nullptr;
    float *dn32 = nullptr;
    int *dexp = nullptr;
    float *Txh32 = nullptr, *Tyh32 = nullptr, *Tzh32 = nullptr, *sq32 = nullptr;
    // Small systems: each lc_pcg_solve / lc_solve_local_then_global call is
    // replayed as one CUDA graph, captured on first use and cached per call
    // signature (the same b, x, parameters and tuning), so that the solve's
    // launches reach the GPU together instead of one host call at a time.
    struct GraphSlot {
        bool valid = false;
        unsigned char key[sizeof(lc_params) + 4 * sizeof(void *) + 16] = {};
        size_t keylen = 0;
        cudaGraphExec_t exec = nullptr;
        long long launches = 0;   // kernels in the graph
    };
    int64_t graph_max_cells = 65536;   // 0: never
    GraphSlot gslot[2];                // [0] lc_pcg_solve, [1] lc_solve_local_then_global
    cudaStream_t cap = nullptr;        // private capture stream (created on first use)
    int graph_broken = 0;              // a capture failed: direct launches from then on
    unsigned tuning_gen = 0;           // bumped by every tuning change (part of the key)
};

namespace {

int fail(lc_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int cuda_fail(lc_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, LC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define LC_CUDA(ctx, call)                                           \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);   \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Carve one allocation into aligned pieces.
struct Carver {
    size_t off = 0;
    char *base = nullptr;
    template <class T>
    T *take(size_t count) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T) + 16;
        return p;
    }
};

void carve(lc_op *op, Carver &c) {
    const size_t n = (size_t)op->n, nnz = (size_t)op->nnz;
    const size_t nchunks = (n + lc::kTreeChunk - 1) / lc::kTreeChunk + 2;
    const size_t xblocks = (n + 1023) / 1024 + 2;
    op->ctrl = c.take<lc::Ctrl>(1);
    op->ctrl_loc = c.take<lc::Ctrl>(1);
    op->work = c.take<double>(n);
    op->mask_tmp = c.take<uint8_t>(n);
    op->mask_own = c.take<uint8_t>(n);
    op->tree_a = c.take<double>(nchunks);
    op->tree_b = c.take<double>(nchunks);
    op->ew.blk = c.take<unsigned long long>(xblocks);
    op->ew.nblocks_cap = (int64_t)xblocks;
    op->sub.g2l = c.take<int32_t>(n);
    op->sub.l2g = c.take<int32_t>(n);
    op->sub.rowptr = c.take<int32_t>(n + 1);
    op->sub.col = c.take<int32_t>(nnz);
    op->sub.val = c.take<double>(nnz);
    op->sub.rhs = c.take<double>(n);
    op->sub.xL0 = c.take<double>(n);
    op->sub.K = c.take<int32_t>(1);
    op->sub.nnz = c.take<int32_t>(1);
    op->pw.r = c.take<double>(n);
    op->pw.z = c.take<double>(n);
    op->pw.p0 = c.take<double>(n);
    op->pw.p1 = c.take<double>(n);
    op->pw.q = c.take<double>(n);
    op->pw.e0 = c.take<double>(n);
    op->pw.e1 = c.take<double>(n);
    op->pw.dinv = c.take<double>(n);
    op->pw.partials = c.take<double>((size_t)lc::kMaxGrid * lc::kPartialSlots);
    op->pw.r32 = c.take<float>(n);
    op->pw.z32 = c.take<float>(n);
    op->pw.p032 = c.take<float>(n);
    op->pw.p132 = c.take<float>(n);
    op->pw.q32 = c.take<float>(n);
    op->pw.x32 = c.take<float>(n);
    op->pw.dinv32 = c.take<float>(n);
    op->pw.val32 = c.take<float>(nnz);
    op->pw.xh = c.take<double>(n);
    op->pw.ahat = c.take<double>(nnz);
    if (op->kind == 0) {
        op->dinv = c.take<double>(n);
        op->D32 = c.take<float>(n);
        op->Tx32 = c.take<float>(n);
        op->Ty32 = c.take<float>(n);
        op->Tz32 = op->st.dim == 3 ? c.take<float>(n) : nullptr;
        op->dinv32 = c.take<float>(n);
        op->sc = c.take<double>(n);
        op->sq = c.take<double>(n);
        op->Txh = c.take<double>(n);
        op->Tyh = c.take<double>(n);
        op->Tzh = op->st.dim == 3 ? c.take<double>(n) : nullptr;
        op->dn32 = c.take<float>(n);
        op->dexp = c.take<int>(1);
        op->Txh32 = c.take<float>(n);
        op->Tyh32 = c.take<float>(n);
        op->Tzh32 = op->st.dim == 3 ? c.take<float>(n) : nullptr;
        op->sq32 = c.take<float>(n);
        const size_t words = (size_t)op->st.ny * op->st.nz * lc::bits_words(op->st);
        op->bits_a = c.take<uint32_t>(words);
        op->bits_b = c.take<uint32_t>(words);
    }
}

int alloc_op(lc_op *op) {
    Carver probe;
    carve(op, probe);
    void *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, probe.off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(op->ctx, LC_ERR_NO_MEMORY, "workspace of %zu bytes: %s", probe.off, cudaGetErrorString(e));
    }
    op->arena = mem;
    Carver real;
    real.base = static_cast<char *>(mem);
    carve(op, real);
    LC_CUDA(op->ctx, cudaMemset(op->ctrl, 0, sizeof(lc::Ctrl)));
    LC_CUDA(op->ctx, cudaMemset(op->ctrl_loc, 0, sizeof(lc::Ctrl)));
    for (auto &ev : op->ev) LC_CUDA(op->ctx, cudaEventCreate(&ev));
    return LC_OK;
}

lc::Csr sub_csr(const lc_op *op) {
    lc::Csr c{};
    c.n = (int32_t)op->n;
    c.n_dev = op->sub.K;
    c.rp = op->sub.rowptr;
    c.ci = op->sub.col;
    c.av = op->sub.val;
    return c;
}

int check_common(lc_ctx *ctx, const lc_op *op) {
    if (!ctx) return LC_ERR_INVALID_ARG;
    if (!op) return fail(ctx, LC_ERR_INVALID_ARG, "null operator");
    if (op->ctx != ctx) return fail(ctx, LC_ERR_INVALID_ARG, "operator belongs to another context");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return LC_OK;
}

// Threshold / expansion of an already computed r (or g) in op->work or r.
int run_threshold_expand(lc_ctx *ctx, const lc_op *op, const double *v, const double *x0, int exp_mode, int rounds,
                         uint8_t *mask, cudaStream_t s) {
    uint8_t *tmp = op->mask_tmp;
    if (op->kind == 0) {
        if (exp_mode == LC_EXP_DILATE && rounds > 0) {
            LC_CUDA(ctx, lc::launch_threshold_dilate_bits(op->st, v, rounds, mask, op->bits_a, op->bits_b, op->ctrl,
                                                          s));
            return LC_OK;
        }
        if (exp_mode == LC_EXP_PAPER && rounds > 0) {
            uint8_t *cur = (rounds % 2 == 0) ? mask : tmp;
            LC_CUDA(ctx, lc::launch_threshold_dilate_bits(op->st, v, 0, cur, op->bits_a, op->bits_b, op->ctrl, s));
            for (int m = 0; m < rounds; ++m) {
                uint8_t *nxt = cur == mask ? tmp : mask;
                LC_CUDA(ctx, lc::launch_expand_paper_stencil(op->st, v, x0, m, cur, nxt, op->ctrl, s));
                cur = nxt;
            }
            return LC_OK;
        }
        LC_CUDA(ctx, lc::launch_threshold_dilate_bits(op->st, v, 0, mask, op->bits_a, op->bits_b, op->ctrl, s));
        return LC_OK;
    }
    const int32_t n = (int32_t)op->n;
    if (rounds <= 0 || exp_mode == LC_EXP_NONE) {
        LC_CUDA(ctx, lc::launch_threshold_csr(n, v, mask, op->ctrl, s));
        return LC_OK;
    }
    uint8_t *cur = (rounds % 2 == 0) ? mask : tmp;
    LC_CUDA(ctx, lc::launch_threshold_csr(n, v, cur, op->ctrl, s));
    for (int m = 0; m < rounds; ++m) {
        uint8_t *nxt = cur == mask ? tmp : mask;
        if (exp_mode == LC_EXP_DILATE) LC_CUDA(ctx, lc::launch_dilate_csr(op->csr, cur, nxt, s));
        else LC_CUDA(ctx, lc::launch_expand_paper_csr(op->csr, v, x0, m, cur, nxt, op->ctrl, s));
        cur = nxt;
    }
    return LC_OK;
}

int mark_residual_impl(lc_ctx *ctx, const lc_op *op, const double *b, const double *x0, const lc_mark_params *p,
                       uint8_t *mask, double *r0, int32_t *K_dev, double *tau_dev, cudaStream_t s) {
    if (!b || !x0 || !p || !mask) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if (p->thr_mode != LC_THR_EPS_NORMB && p->thr_mode != LC_THR_REL_MAX)
        return fail(ctx, LC_ERR_INVALID_ARG, "unknown threshold mode %d", p->thr_mode);
    if (!(p->thr_param >= 0.0) || !std::isfinite(p->thr_param))
        return fail(ctx, LC_ERR_INVALID_ARG, "threshold parameter must be finite and >= 0");
    if (p->exp_mode < LC_EXP_NONE || p->exp_mode > LC_EXP_PAPER)
        return fail(ctx, LC_ERR_INVALID_ARG, "unknown expansion mode %d", p->exp_mode);
    if (p->exp_rounds < 0 || p->exp_rounds > lc::kMaxExpRounds)
        return fail(ctx, LC_ERR_INVALID_ARG, "expansion rounds must be in [0, %d]", lc::kMaxExpRounds);
    double *r = r0 ? r0 : op->work;
    const double param = p->thr_param == 0.0 ? 0.0 : p->thr_param;   // no -0
    LC_CUDA(ctx, cudaMemsetAsync(op->ctrl, 0, sizeof(lc::Ctrl), s));
    const int tree = p->thr_mode == LC_THR_EPS_NORMB;
    if (op->kind == 0) LC_CUDA(ctx, lc::launch_residual_stencil(op->st, b, x0, r, tree, op->tree_a, op->ctrl, s));
    else LC_CUDA(ctx, lc::launch_residual_csr(op->csr, b, x0, r, tree, op->tree_a, op->ctrl, s));
    if (tree) {
        const int64_t nchunks = (op->n + lc::kTreeChunk - 1) / lc::kTreeChunk;
        LC_CUDA(ctx, lc::launch_tree_finish(op->tree_a, op->tree_b, nchunks, op->n, param, op->ctrl, tau_dev, s));
    } else {
        LC_CUDA(ctx, lc::launch_tau_relmax(param, op->ctrl, tau_dev, s));
    }
    int rc = run_threshold_expand(ctx, op, r, x0, p->exp_mode, p->exp_rounds, mask, s);
    if (rc) return rc;
    LC_CUDA(ctx, cudaMemsetAsync(&op->ctrl->K, 0, sizeof(int32_t), s));
    LC_CUDA(ctx, lc::launch_count_mask(op->n, mask, op->ctrl, K_dev, s));
    return LC_OK;
}

int mark_gradient_impl(lc_ctx *ctx, const lc_op *op, const double *x0, double alpha, int32_t layers, uint8_t *mask,
                       int32_t *K_dev, double *gmax_dev, cudaStream_t s) {
    if (!x0 || !mask) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(ctx, LC_ERR_INVALID_ARG, "alpha must be in [0, 1]");
    if (layers < 0 || layers > lc::kMaxExpRounds)
        return fail(ctx, LC_ERR_INVALID_ARG, "layers must be in [0, %d]", lc::kMaxExpRounds);
    LC_CUDA(ctx, cudaMemsetAsync(op->ctrl, 0, sizeof(lc::Ctrl), s));
    if (op->kind == 0) LC_CUDA(ctx, lc::launch_gradient_stencil(op->st, x0, op->work, op->ctrl, s));
    else LC_CUDA(ctx, lc::launch_gradient_csr(op->csr, x0, op->work, op->ctrl, s));
    LC_CUDA(ctx, lc::launch_gmax_threshold(alpha == 0.0 ? 0.0 : alpha, op->ctrl, gmax_dev, s));
    int rc = run_threshold_expand(ctx, op, op->work, x0, layers > 0 ? LC_EXP_DILATE : LC_EXP_NONE, layers, mask, s);
    if (rc) return rc;
    LC_CUDA(ctx, cudaMemsetAsync(&op->ctrl->K, 0, sizeof(int32_t), s));
    LC_CUDA(ctx, lc::launch_count_mask(op->n, mask, op->ctrl, K_dev, s));
    return LC_OK;
}

int extract_impl(lc_ctx *ctx, const lc_op *op, const uint8_t *mask, const double *b, const double *x0,
                 const lc_subsys &out, cudaStream_t s) {
    if (!mask || !b || !x0) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if (!out.g2l || !out.l2g || !out.rowptr || !out.col || !out.val || !out.rhs || !out.xL0 || !out.K || !out.nnz)
        return fail(ctx, LC_ERR_INVALID_ARG, "null subsystem output");
    lc::ExtractWork w = op->ew;
    if (op->kind == 0) LC_CUDA(ctx, lc::launch_extract_stencil(op->st, mask, b, x0, out, w, op->ctrl, s));
    else LC_CUDA(ctx, lc::launch_extract_csr(op->csr, mask, b, x0, out, w, op->ctrl, s));
    return LC_OK;
}

int check_solve_params(lc_ctx *ctx, const lc_solve_params *p) {
    if (!p) return fail(ctx, LC_ERR_INVALID_ARG, "null solve parameters");
    if (!(p->tol >= 0.0) || !std::isfinite(p->tol)) return fail(ctx, LC_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (p->max_iter < 0) return fail(ctx, LC_ERR_INVALID_ARG, "max_iter < 0");
    if (p->precision == LC_PREC_MIXED) {
        if (!(p->inner_tol > 0.0 && p->inner_tol < 1.0))
            return fail(ctx, LC_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
        if (p->max_outer < 1) return fail(ctx, LC_ERR_INVALID_ARG, "max_outer must be >= 1");
    } else if (p->precision != LC_PREC_FP64) {
        return fail(ctx, LC_ERR_INVALID_ARG, "unknown precision %d", p->precision);
    }
    return LC_OK;
}

int pcg_impl(lc_ctx *ctx, const lc_op *op, const double *b, double *x, const lc_solve_params *p, lc::Ctrl *ctrl,
             bool local, cudaStream_t s) {
    lc::PcgArgs a{b,           x,           p->tol,        p->max_iter,  3,
                  op->pcg_minblocks, p->precision, p->inner_tol, p->max_outer, op->pcg_scaled, op->pcg_wide,
                  op->pcg_big, op->pcg_pairdot, op->pcg_lazy_x, op->csr_store_p};
    lc::PcgWork w = op->pw;
    LC_CUDA(ctx, cudaMemsetAsync(&ctrl->status, 0, sizeof(int32_t), s));
    if (local) {
        // the local system is small and its barriers dominate: one thread-block
        // cluster when it fits (FP64), else one block per SM
        const bool cl = op->local_cluster_rows > 0 && p->precision == LC_PREC_FP64 && lc::cluster_local_rows() > 0;
        if (cl)
            LC_CUDA(ctx, lc::launch_pcg_csr_cluster(sub_csr(op), a, op->local_cluster_rows, op->local_cluster_threads,
                                                    op->local_cluster_ctas, ctrl, s));
        const int cap = op->local_grid_cap > 0 ? op->local_grid_cap : ctx->sms;
        if (op->local_pipelined)   // FP64, or FP32 inner solves in FP64 refinement
            LC_CUDA(ctx, lc::launch_pcg_csr_pipelined(sub_csr(op), a, w, ctrl, cap, s, cl));
        else if (op->local_single && p->precision == LC_PREC_FP64)
            LC_CUDA(ctx, lc::launch_pcg_csr_single(sub_csr(op), a, w, ctrl, cap, s, cl));
        else
            LC_CUDA(ctx, lc::launch_pcg_csr(sub_csr(op), a, w, ctrl, cap, s, cl));
    } else if (op->kind == 0) {
        LC_CUDA(ctx, lc::launch_pcg_stencil(op->st, a, w, ctrl, op->pcg_grid_cap, s));
    } else {
        LC_CUDA(ctx, lc::launch_pcg_csr(op->csr, a, w, ctrl, op->pcg_grid_cap, s));
    }
    return LC_OK;
}

int read_ctrl(lc_ctx *ctx, const lc::Ctrl *dev, lc::Ctrl *host) {
    LC_CUDA(ctx, cudaMemcpy(host, dev, sizeof(lc::Ctrl), cudaMemcpyDeviceToHost));
    return LC_OK;
}

int status_of(const lc::Ctrl &c) {
    if (c.status != LC_OK) return c.status;
    if (c.converged == -1) return LC_ERR_BREAKDOWN;
    if (c.converged == 0) return LC_ERR_NOT_CONVERGED;
    return LC_OK;
}

}  // namespace

extern "C" {

const char *lc_error_string(int code) {
    switch (code) {
        case LC_OK: return "ok";
        case LC_ERR_INVALID_ARG: return "invalid argument";
        case LC_ERR_CUDA: return "CUDA error";
        case LC_ERR_NO_MEMORY: return "out of device memory";
        case LC_ERR_NOT_CONVERGED: return "not converged";
        case LC_ERR_BREAKDOWN: return "Krylov breakdown (operator not SPD or non-finite data)";
        case LC_ERR_TIMEOUT: return "grid-wide wait timed out";
        case LC_ERR_TOO_LARGE: return "problem too large";
        case LC_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown error";
    }
}

const char *lc_last_error(const lc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t lc_kernel_launch_count(void) { return (int64_t)lc::g_launches.load(std::memory_order_relaxed); }

int lc_checked_selftest(void *stream) {
#ifndef LC_CHECKED
    (void)stream;
    return LC_ERR_UNSUPPORTED;
#else
    lc::checked_selftest_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(4);
    lc::note_launches(1);
    return cudaGetLastError() == cudaSuccess ? LC_OK : LC_ERR_CUDA;
#endif
}

int lc_checked_status(int32_t *failures, char *where, int32_t len) {
    if (failures) *failures = 0;
    if (where && len > 0) where[0] = 0;
#ifndef LC_CHECKED
    if (where && len > 0) snprintf(where, (size_t)len, "not a bounds-checked build");
    return LC_ERR_UNSUPPORTED;
#else
    std::lock_guard<std::mutex> g(lc::g_check_mu);
    int32_t bad = 0;
    for (const auto &u : lc::check_units()) {
        const unsigned line = u.first();
        if (!line) continue;
        if (!bad && where && len > 0) {
            const char *base = strrchr(u.second, '/');
            snprintf(where, (size_t)len, "%s:%u", base ? base + 1 : u.second, line);
        }
        ++bad;
    }
    if (failures) *failures = bad;
    return LC_OK;
#endif
}

int lc_assemble_diffusion_2d(lc_ctx *ctx, const int32_t shape[2], const double *k, double dt, double *D,
                             double *Tx, double *Ty, void *stream) {
    if (!ctx) return LC_ERR_INVALID_ARG;
    if (!shape || !k || !D || !Tx || !Ty) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if (shape[0] <= 0 || shape[1] <= 0) return fail(ctx, LC_ERR_INVALID_ARG, "shape must be positive");
    if ((int64_t)shape[0] * shape[1] >= (int64_t)INT32_MAX) return fail(ctx, LC_ERR_TOO_LARGE, "N does not fit int32");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, LC_ERR_INVALID_ARG, "dt must be finite and > 0");
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    LC_CUDA(ctx, lc::launch_assemble_2d(shape[0], shape[1], k, dt, D, Tx, Ty, (cudaStream_t)stream));
    return LC_OK;
}

int lc_op_refresh(lc_op *op, void *stream) {
    if (!op) return LC_ERR_INVALID_ARG;
    if (op->kind != 0) return LC_OK;
    LC_CUDA(op->ctx, cudaSetDevice(op->ctx->device));
    LC_CUDA(op->ctx, lc::launch_dinv_stencil(op->n, op->st.D, op->dinv, op->D32, op->st.Tx, op->st.Ty, op->st.Tz,
                                             op->Tx32, op->Ty32, op->Tz32, op->dinv32, (cudaStream_t)stream));
    if (op->st.sc)
        LC_CUDA(op->ctx, lc::launch_scaling(op->st, op->sc, op->sq, op->Txh, op->Tyh, op->Tzh, op->dn32, op->dexp,
                                            op->Txh32, op->Tyh32, op->Tzh32, op->sq32, (cudaStream_t)stream));
    return LC_OK;
}

int lc_adjoint_grad_k_2d(lc_ctx *ctx, const int32_t shape[2], const double *k, const double *x, const double *lam,
                         double *dk, void *stream) {
    if (!ctx) return LC_ERR_INVALID_ARG;
    if (!shape || !k || !x || !lam || !dk) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if (shape[0] <= 0 || shape[1] <= 0) return fail(ctx, LC_ERR_INVALID_ARG, "shape must be positive");
    if ((int64_t)shape[0] * shape[1] >= (int64_t)INT32_MAX) return fail(ctx, LC_ERR_TOO_LARGE, "N does not fit int32");
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    LC_CUDA(ctx, lc::launch_adjoint_grad_k_2d(shape[0], shape[1], k, x, lam, dk, (cudaStream_t)stream));
    return LC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batched Alg 1

struct lc_batch {
    lc_ctx *ctx = nullptr;
    int32_t nsys = 0;
    int64_t cells = 0;
    void *arena = nullptr;
    lc::BatchLaunch L{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int32_t> nx, ny;
};

namespace {

void batch_carve(lc_batch *bt, Carver &c) {
    const size_t T = (size_t)bt->cells, S = (size_t)bt->nsys;
    lc::BatchView &v = bt->L.v;
    v.nx = c.take<int32_t>(S);
    v.ny = c.take<int32_t>(S);
    v.off = c.take<int64_t>(S);
    v.order = c.take<int32_t>(S);
    v.next = c.take<int32_t>(2);
    v.stat_i = c.take<int32_t>(8 * S);
    v.stat_d = c.take<double>(4 * S);
    v.D32 = c.take<float>(T);
    v.Tx32 = c.take<float>(T);
    v.Ty32 = c.take<float>(T);
    v.dinv32 = c.take<float>(T);
    v.r = c.take<double>(T);
    v.m0 = c.take<uint8_t>(T);
    v.m1 = c.take<uint8_t>(T);
    v.g2l = c.take<int32_t>(T);
    v.l2g = c.take<int32_t>(T);
    v.rowptr = c.take<int32_t>(T + S);
    v.col = c.take<int32_t>(5 * T);
    v.val = c.take<double>(5 * T);
    v.val32 = c.take<float>(5 * T);
    v.rhs = c.take<double>(T);
    v.xl = c.take<double>(T);
    v.dl32 = c.take<float>(T);
    v.r32 = c.take<float>(T);
    v.z32 = c.take<float>(T);
    v.p32 = c.take<float>(T);
    v.q32 = c.take<float>(T);
    v.d32 = c.take<float>(T);
}

int batch_params(lc_ctx *ctx, const lc_params *p, lc::BatchParams &bp) {
    if (!p) return fail(ctx, LC_ERR_INVALID_ARG, "null parameters");
    if (p->mark_mode != LC_MARK_RESIDUAL || p->mark.thr_mode != LC_THR_REL_MAX ||
        (p->mark.exp_mode != LC_EXP_NONE && p->mark.exp_mode != LC_EXP_DILATE) ||
        p->global.precision != LC_PREC_MIXED || p->local.precision != LC_PREC_MIXED || p->gs_sweeps != 0)
        return fail(ctx, LC_ERR_UNSUPPORTED,
                    "batched solve: residual marking with the relative threshold and dilation, mixed precision");
    if (!(p->mark.thr_param >= 0.0) || !std::isfinite(p->mark.thr_param) || p->mark.exp_rounds < 0 ||
        p->mark.exp_rounds > lc::kMaxExpRounds)
        return fail(ctx, LC_ERR_INVALID_ARG, "bad marking parameters");
    int rc;
    if ((rc = check_solve_params(ctx, &p->global)) || (rc = check_solve_params(ctx, &p->local))) return rc;
    bp.beta = p->mark.thr_param == 0.0 ? 0.0 : p->mark.thr_param;
    bp.layers = p->mark.exp_mode == LC_EXP_DILATE ? p->mark.exp_rounds : 0;
    bp.tol = p->global.tol;
    bp.tol_local = p->local.tol;
    bp.inner_tol = p->global.inner_tol;
    bp.max_outer = p->global.max_outer;
    bp.max_inner = p->global.max_iter;
    return LC_OK;
}

}  // namespace

namespace {

// Runs enqueue(stream) -- a solve's whole sequence of stream-ordered work --
// directly, or, for operators of at most graph_max_cells cells, as a cached
// CUDA graph: captured on a private stream the first time a call signature
// (key) is seen and replayed on `s` afterwards.  Every decision of the
// sequence that depends on data is taken on the device, so a replay does
// what a direct call does; kernel sizes depend only on the operator, the
// parameters and the tuning, all of which are in the key.  If a capture
// fails (an operation the graph cannot hold), the operator runs its calls
// directly from then on.
template <class F>
int run_graphed(lc_ctx *ctx, lc_op *op, int slot, const void *key, size_t keylen, cudaStream_t s, F enqueue) {
    if (op->n > op->graph_max_cells || op->graph_broken || keylen > sizeof(op->gslot[0].key)) return enqueue(s, false);
    lc_op::GraphSlot &g = op->gslot[slot];
    if (!(g.valid && g.keylen == keylen && memcmp(g.key, key, keylen) == 0)) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        g.valid = false;
        if (!op->cap && cudaStreamCreateWithFlags(&op->cap, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            op->graph_broken = 1;
            return enqueue(s, false);
        }
        if (cudaStreamBeginCapture(op->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            op->graph_broken = 1;
            return enqueue(s, false);
        }
        const long long l0 = lc::g_launches.load(std::memory_order_relaxed);
        const int rc = enqueue(op->cap, true);
        const long long nl = lc::g_launches.load(std::memory_order_relaxed) - l0;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(op->cap, &graph);
        if (rc == LC_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        lc::g_launches.fetch_sub(nl, std::memory_order_relaxed);   // counted when the graph runs
        if (rc != LC_OK || e != cudaSuccess || !g.exec) {
            cudaGetLastError();
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            if (rc != LC_OK && rc != LC_ERR_CUDA) return rc;   // an argument error, not the capture's
            op->graph_broken = 1;
            return enqueue(s, false);
        }
        memcpy(g.key, key, keylen);
        g.keylen = keylen;
        g.launches = nl;
        g.valid = true;
    }
    LC_CUDA(ctx, cudaGraphLaunch(g.exec, s));
    lc::g_launches.fetch_add(g.launches, std::memory_order_relaxed);
    return LC_OK;
}

// An event of the stats: inside a capture it must become a node of the graph
// (an external record), else the replay would not record it.
cudaError_t record(cudaEvent_t ev, cudaStream_t q, bool capturing) {
    return cudaEventRecordWithFlags(ev, q, capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// Milliseconds between two recorded events (0, and the error cleared, if the
// runtime cannot time them).
float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        ms = 0.f;
    }
    return ms;
}

// the signature of a solve call, for run_graphed
template <class P>
size_t call_key(unsigned char *k, const lc_op *op, const void *b, const void *x, const P *p, bool stats) {
    size_t n = 0;
    const auto put = [&](const void *v, size_t sz) { memcpy(k + n, v, sz); n += sz; };
    put(&b, sizeof b);
    put(&x, sizeof x);
    put(p, sizeof *p);
    const unsigned char st = stats ? 1 : 0;
    put(&st, 1);
    put(&op->tuning_gen, sizeof op->tuning_gen);
    return n;
}

}  // namespace

extern "C" {

int lc_batch_create(lc_ctx *ctx, lc_batch **out, int32_t nsys, const int32_t *nx, const int32_t *ny, const double *D,
                    const double *Tx, const double *Ty) {
    if (!ctx || !out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    if (nsys <= 0 || !nx || !ny || !D || !Tx || !Ty) return fail(ctx, LC_ERR_INVALID_ARG, "bad batch description");
    int64_t cells = 0;
    std::vector<int64_t> off(nsys);
    for (int32_t s = 0; s < nsys; ++s) {
        if (nx[s] <= 0 || ny[s] <= 0) return fail(ctx, LC_ERR_INVALID_ARG, "system %d has a non-positive shape", s);
        off[s] = cells;
        cells += (int64_t)nx[s] * ny[s];
    }
    if (5 * cells + nsys >= (int64_t)INT32_MAX || (int64_t)nx[0] * ny[0] >= (int64_t)INT32_MAX)
        return fail(ctx, LC_ERR_TOO_LARGE, "batch of %lld cells exceeds int32 indexing", (long long)cells);
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    lc_batch *bt = new (std::nothrow) lc_batch;
    if (!bt) return LC_ERR_NO_MEMORY;
    bt->ctx = ctx;
    ctx_ref(ctx);
    bt->nsys = nsys;
    bt->cells = cells;
    bt->nx.assign(nx, nx + nsys);
    bt->ny.assign(ny, ny + nsys);
    Carver probe;
    batch_carve(bt, probe);
    if (cudaMalloc(&bt->arena, probe.off) != cudaSuccess) {
        cudaGetLastError();
        bt->arena = nullptr;
        lc_batch_destroy(bt);
        return fail(ctx, LC_ERR_NO_MEMORY, "batch workspace of %zu bytes", probe.off);
    }
    Carver real;
    real.base = static_cast<char *>(bt->arena);
    batch_carve(bt, real);
    lc::BatchView &v = bt->L.v;
    v.nsys = nsys;
    v.D = D; v.Tx = Tx; v.Ty = Ty;
    std::vector<int32_t> order(nsys);
    for (int32_t s = 0; s < nsys; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return (int64_t)nx[a] * ny[a] > (int64_t)nx[b] * ny[b];
    });
    cudaError_t e = cudaMemcpy(const_cast<int32_t *>(v.nx), nx, sizeof(int32_t) * nsys, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(const_cast<int32_t *>(v.ny), ny, sizeof(int32_t) * nsys, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(const_cast<int64_t *>(v.off), off.data(), sizeof(int64_t) * nsys, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(const_cast<int32_t *>(v.order), order.data(), sizeof(int32_t) * nsys, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = lc::launch_batch_f32(cells, D, Tx, Ty, const_cast<float *>(v.D32), const_cast<float *>(v.Tx32),
                                 const_cast<float *>(v.Ty32), const_cast<float *>(v.dinv32), 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        int rc = cuda_fail(ctx, e, "batch set-up");
        lc_batch_destroy(bt);
        return rc;
    }
    bt->L.block = 512;
    bt->L.ctas_per_sm = 0;
    bt->L.cluster = 1;
    bt->L.big_cells = 65536;
    *out = bt;
    return LC_OK;
}

int lc_batch_destroy(lc_batch *bt) {
    if (!bt) return LC_OK;
    if (bt->ctx) cudaSetDevice(bt->ctx->device);
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    if (bt->arena) cudaFree(bt->arena);
    lc_ctx *ctx = bt->ctx;
    delete bt;
    ctx_unref(ctx);
    return LC_OK;
}

// systems solved by whole clusters: those of at least big_cells cells (the
// queue is sorted by size, largest first)
static void batch_split(lc_batch *bt) {
    int32_t nbig = 0;
    if (bt->L.cluster > 1)
        for (int32_t s = 0; s < bt->nsys; ++s)
            if ((int64_t)bt->nx[s] * bt->ny[s] >= bt->L.big_cells) ++nbig;
    bt->L.v.nbig = nbig;
}

static int batch_enqueue(lc_batch *bt, cudaStream_t s) {
    lc_ctx *ctx = bt->ctx;
    batch_split(bt);
    LC_CUDA(ctx, cudaMemsetAsync(bt->L.v.next, 0, 2 * sizeof(int32_t), s));
    LC_CUDA(ctx, lc::launch_batched(&bt->L, ctx->sms, s));
    return LC_OK;
}

int lc_batch_solve(lc_ctx *ctx, lc_batch *bt, const double *b, double *x, const lc_params *p, void *stream) {
    if (!ctx || !bt || bt->ctx != ctx) return LC_ERR_INVALID_ARG;
    if (!b || !x) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    int rc;
    if ((rc = batch_params(ctx, p, bt->L.p))) return rc;
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    bt->L.v.b = b;
    bt->L.v.x = x;
    return batch_enqueue(bt, (cudaStream_t)stream);
}

int lc_batch_capture(lc_ctx *ctx, lc_batch *bt, const double *b, double *x, const lc_params *p) {
    if (!ctx || !bt || bt->ctx != ctx) return LC_ERR_INVALID_ARG;
    if (!b || !x) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    int rc;
    if ((rc = batch_params(ctx, p, bt->L.p))) return rc;
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    bt->L.v.b = b;
    bt->L.v.x = x;
    if (bt->exec) { cudaGraphExecDestroy(bt->exec); bt->exec = nullptr; }
    if (bt->graph) { cudaGraphDestroy(bt->graph); bt->graph = nullptr; }
    cudaStream_t cs;
    LC_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = batch_enqueue(bt, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (!rc && e2 == cudaSuccess) {
            bt->graph = g;
            e = cudaGraphInstantiate(&bt->exec, g, 0);
        } else {
            e = e2;
            if (g) cudaGraphDestroy(g);
        }
    }
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch graph capture");
    return LC_OK;
}

int lc_batch_replay(lc_batch *bt, void *stream) {
    if (!bt) return LC_ERR_INVALID_ARG;
    if (!bt->exec) return fail(bt->ctx, LC_ERR_INVALID_ARG, "no captured graph (call lc_batch_capture first)");
    LC_CUDA(bt->ctx, cudaSetDevice(bt->ctx->device));
    LC_CUDA(bt->ctx, cudaGraphLaunch(bt->exec, (cudaStream_t)stream));
    lc::note_launches(1);
    return LC_OK;
}

int lc_batch_stats(lc_batch *bt, lc_stats *per_system, void *stream) {
    if (!bt || !per_system) return LC_ERR_INVALID_ARG;
    LC_CUDA(bt->ctx, cudaSetDevice(bt->ctx->device));
    LC_CUDA(bt->ctx, cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<int32_t> si(8 * (size_t)bt->nsys);
    std::vector<double> sd(4 * (size_t)bt->nsys);
    LC_CUDA(bt->ctx, cudaMemcpy(si.data(), bt->L.v.stat_i, sizeof(int32_t) * si.size(), cudaMemcpyDeviceToHost));
    LC_CUDA(bt->ctx, cudaMemcpy(sd.data(), bt->L.v.stat_d, sizeof(double) * sd.size(), cudaMemcpyDeviceToHost));
    int worst = LC_OK;
    for (int32_t s = 0; s < bt->nsys; ++s) {
        lc_stats &st = per_system[s];
        memset(&st, 0, sizeof st);
        st.status = si[8 * s + 0];
        st.n = bt->nx[s] * bt->ny[s];
        st.K = si[8 * s + 1];
        st.nnzB = si[8 * s + 2];
        st.it_local = si[8 * s + 3];
        st.it_global = si[8 * s + 4];
        st.restarts = si[8 * s + 6];
        st.early_exit = si[8 * s + 7];
        st.tau = sd[4 * s + 0];
        st.relres_tilde = sd[4 * s + 1];
        st.relres_final = sd[4 * s + 2];
        st.eta = st.n ? (double)st.K / st.n : 0.0;
        if (st.status != LC_OK && worst == LC_OK) worst = st.status;
    }
    return worst;
}

int lc_batch_domain(lc_batch *bt, int32_t sys, uint8_t *mask, int32_t *g2l, int32_t *l2g, int32_t *rowptr,
                    int32_t *col, double *val, double *rhs, void *stream) {
    if (!bt) return LC_ERR_INVALID_ARG;
    if (sys < 0 || sys >= bt->nsys) return fail(bt->ctx, LC_ERR_INVALID_ARG, "system index out of range");
    lc_ctx *ctx = bt->ctx;
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    LC_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
    const lc::BatchView &v = bt->L.v;
    int64_t off = 0;
    for (int32_t t = 0; t < sys; ++t) off += (int64_t)bt->nx[t] * bt->ny[t];
    const size_t n = (size_t)bt->nx[sys] * bt->ny[sys];
    int32_t kn[2];   // K, nnz(B) of the last solve
    LC_CUDA(ctx, cudaMemcpy(kn, v.stat_i + 8 * (int64_t)sys + 1, sizeof kn, cudaMemcpyDeviceToHost));
    const size_t K = (size_t)kn[0], nz = (size_t)kn[1];
    // after `layers` dilation rounds the batched kernel's mask is in m0 for an even count, else m1
    const uint8_t *m = (bt->L.p.layers % 2 == 0) ? v.m0 : v.m1;
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    if (mask) LC_CUDA(ctx, cudaMemcpy(mask, m + off, n, dd));
    if (g2l) LC_CUDA(ctx, cudaMemcpy(g2l, v.g2l + off, sizeof(int32_t) * n, dd));
    if (l2g && K) LC_CUDA(ctx, cudaMemcpy(l2g, v.l2g + off, sizeof(int32_t) * K, dd));
    if (rowptr) LC_CUDA(ctx, cudaMemcpy(rowptr, v.rowptr + off + sys, sizeof(int32_t) * (K + 1), dd));
    if (col && nz) LC_CUDA(ctx, cudaMemcpy(col, v.col + 5 * off, sizeof(int32_t) * nz, dd));
    if (val && nz) LC_CUDA(ctx, cudaMemcpy(val, v.val + 5 * off, sizeof(double) * nz, dd));
    if (rhs && K) LC_CUDA(ctx, cudaMemcpy(rhs, v.rhs + off, sizeof(double) * K, dd));
    return LC_OK;
}

int lc_batch_set_tuning(lc_batch *bt, const char *key, int32_t value) {
    if (!bt || !key) return LC_ERR_INVALID_ARG;
    if (!strcmp(key, "block")) {
        if (value != 256 && value != 512 && value != 1024)
            return fail(bt->ctx, LC_ERR_INVALID_ARG, "block must be 256, 512 or 1024");
        bt->L.block = value;
        return LC_OK;
    }
    if (!strcmp(key, "ctas_per_sm")) {
        if (value < 0 || value > 32) return fail(bt->ctx, LC_ERR_INVALID_ARG, "ctas_per_sm must be 0..32");
        bt->L.ctas_per_sm = value;
        return LC_OK;
    }
    if (!strcmp(key, "cluster")) {
        if (value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
            return fail(bt->ctx, LC_ERR_INVALID_ARG, "cluster must be 1, 2, 4, 8 or 16");
        bt->L.cluster = value;
        return LC_OK;
    }
    if (!strcmp(key, "big_cells")) {
        if (value < 1) return fail(bt->ctx, LC_ERR_INVALID_ARG, "big_cells must be >= 1");
        bt->L.big_cells = value;
        return LC_OK;
    }
    return fail(bt->ctx, LC_ERR_INVALID_ARG, "unknown tuning key '%s'", key);
}

int lc_op_set_tuning(lc_op *op, const char *key, int32_t value) {
    if (!op || !key) return LC_ERR_INVALID_ARG;
    ++op->tuning_gen;
    if (!strcmp(key, "graph_max_cells")) {
        if (value < 0) return fail(op->ctx, LC_ERR_INVALID_ARG, "graph_max_cells must be >= 0");
        op->graph_max_cells = value;
        return LC_OK;
    }
    if (!strcmp(key, "pcg_minblocks")) {
        if (value < 1 || value > 4) return fail(op->ctx, LC_ERR_INVALID_ARG, "pcg_minblocks must be 1..4");
        op->pcg_minblocks = value;
        return LC_OK;
    }
    if (!strcmp(key, "pcg_grid_cap")) {
        if (value < 0 || value > lc::kMaxGrid) return fail(op->ctx, LC_ERR_INVALID_ARG, "pcg_grid_cap out of range");
        op->pcg_grid_cap = value;
        return LC_OK;
    }
    if (!strcmp(key, "pcg_scaled")) {
        if (value < 0 || value > 1) return fail(op->ctx, LC_ERR_INVALID_ARG, "pcg_scaled must be 0 or 1");
        op->pcg_scaled = value;
        return LC_OK;
    }
    if (!strcmp(key, "local_cluster_rows")) {
        if (value < 0) return fail(op->ctx, LC_ERR_INVALID_ARG, "local_cluster_rows must be >= 0");
        op->local_cluster_rows = value;
        return LC_OK;
    }
    if (!strcmp(key, "pcg_lazy_x")) {
        if (value < 0 || value > 1) return fail(op->ctx, LC_ERR_INVALID_ARG, "pcg_lazy_x must be 0 or 1");
        op->pcg_lazy_x = value;
        return LC_OK;
    }
    if (!strcmp(key, "csr_store_p")) {
        if (value < 0 || value > 1) return fail(op->ctx, LC_ERR_INVALID_ARG, "csr_store_p must be 0 or 1");
        op->csr_store_p = value;
        return LC_OK;
    }
    if (!strcmp(key, "local_grid_cap")) {
        if (value < 0 || value > lc::kMaxGrid) return fail(op->ctx, LC_ERR_INVALID_ARG, "local_grid_cap out of range");
        op->local_grid_cap = value;
        return LC_OK;
    }
    if (!strcmp(key, "pcg_pairdot")) {
        if (value < 0 || value > 1) return fail(op->ctx, LC_ERR_INVALID_ARG, "pcg_pairdot must be 0 or 1");
        op->pcg_pairdot = value;
        return LC_OK;
    }
    if (!strcmp(key, "pcg_big")) {
        if (value < 0 || value > 1) return fail(op->ctx, LC_ERR_INVALID_ARG, "pcg_big must be 0 or 1");
        op->pcg_big = value;
        return LC_OK;
    }
    if (!strcmp(key, "pcg_wide")) {
        if (value < 0 || value > 1) return fail(op->ctx, LC_ERR_INVALID_ARG, "pcg_wide must be 0 or 1");
        op->pcg_wide = value;
        return LC_OK;
    }
    if (!strcmp(key, "local_pipelined")) {
        if (value < 0 || value > 1) return fail(op->ctx, LC_ERR_INVALID_ARG, "local_pipelined must be 0 or 1");
        op->local_pipelined = value;
        return LC_OK;
    }
    if (!strcmp(key, "local_single")) {
        if (value < 0 || value > 1) return fail(op->ctx, LC_ERR_INVALID_ARG, "local_single must be 0 or 1");
        op->local_single = value;
        return LC_OK;
    }
    if (!strcmp(key, "local_cluster_ctas")) {
        if (value != 0 && value != 2 && value != 4 && value != 8 && value != 16)
            return fail(op->ctx, LC_ERR_INVALID_ARG, "local_cluster_ctas must be 0, 2, 4, 8 or 16");
        op->local_cluster_ctas = value;
        return LC_OK;
    }
    if (!strcmp(key, "local_cluster_threads")) {
        if (value != 256 && value != 512 && value != 1024)
            return fail(op->ctx, LC_ERR_INVALID_ARG, "local_cluster_threads must be 256, 512 or 1024");
        op->local_cluster_threads = value;
        return LC_OK;
    }
    return fail(op->ctx, LC_ERR_INVALID_ARG, "unknown tuning key '%s'", key);
}

int lc_op_get_tuning(const lc_op *op, const char *key, int32_t *value) {
    if (!op || !key || !value) return LC_ERR_INVALID_ARG;
    if (!strcmp(key, "pcg_minblocks")) { *value = op->pcg_minblocks; return LC_OK; }
    if (!strcmp(key, "pcg_grid_cap")) { *value = op->pcg_grid_cap; return LC_OK; }
    if (!strcmp(key, "pcg_scaled")) { *value = op->pcg_scaled; return LC_OK; }
    if (!strcmp(key, "local_cluster_rows")) { *value = op->local_cluster_rows; return LC_OK; }
    if (!strcmp(key, "local_cluster_threads")) { *value = op->local_cluster_threads; return LC_OK; }
    if (!strcmp(key, "local_cluster_ctas")) { *value = op->local_cluster_ctas; return LC_OK; }
    if (!strcmp(key, "local_single")) { *value = op->local_single; return LC_OK; }
    if (!strcmp(key, "local_pipelined")) { *value = op->local_pipelined; return LC_OK; }
    if (!strcmp(key, "pcg_wide")) { *value = op->pcg_wide; return LC_OK; }
    if (!strcmp(key, "pcg_big")) { *value = op->pcg_big; return LC_OK; }
    if (!strcmp(key, "pcg_pairdot")) { *value = op->pcg_pairdot; return LC_OK; }
    if (!strcmp(key, "local_grid_cap")) { *value = op->local_grid_cap; return LC_OK; }
    if (!strcmp(key, "pcg_lazy_x")) { *value = op->pcg_lazy_x; return LC_OK; }
    if (!strcmp(key, "csr_store_p")) { *value = op->csr_store_p; return LC_OK; }
    if (!strcmp(key, "graph_max_cells")) { *value = (int32_t)op->graph_max_cells; return LC_OK; }
    return LC_ERR_INVALID_ARG;
}

int lc_ctx_create(lc_ctx **out, int device) {
    if (!out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return LC_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return LC_ERR_CUDA;
    lc_ctx *c = new (std::nothrow) lc_ctx;
    if (!c) return LC_ERR_NO_MEMORY;
    c->device = device;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return LC_OK;
}

int lc_ctx_destroy(lc_ctx *ctx) {
    ctx_unref(ctx);
    return LC_OK;
}

int lc_op_create_stencil(lc_ctx *ctx, lc_op **out, int32_t dim, const int32_t shape[3], const double *D,
                         const double *Tx, const double *Ty, const double *Tz) {
    if (!ctx || !out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(ctx, LC_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (!shape || !D || !Tx || !Ty || (dim == 3 && !Tz)) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    const int64_t nx = shape[0], ny = shape[1], nz = dim == 3 ? shape[2] : 1;
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(ctx, LC_ERR_INVALID_ARG, "shape must be positive");
    if (dim == 2 && shape[2] != 1 && shape[2] != 0) return fail(ctx, LC_ERR_INVALID_ARG, "shape[2] must be 1 for dim 2");
    const int64_t n = nx * ny * nz;
    if (n >= (int64_t)INT32_MAX) return fail(ctx, LC_ERR_TOO_LARGE, "N = %lld does not fit int32", (long long)n);
    const int64_t nnz = n + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1));
    if (nnz >= (int64_t)INT32_MAX) return fail(ctx, LC_ERR_TOO_LARGE, "nnz does not fit int32");
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    lc_op *op = new (std::nothrow) lc_op;
    if (!op) return LC_ERR_NO_MEMORY;
    op->ctx = ctx;
    ctx_ref(ctx);
    op->kind = 0;
    op->n = n;
    op->nnz = nnz;
    op->st.dim = dim;
    op->pcg_minblocks = 3;   // measured best register budget (2D strips and 3D tiles)
    op->st.nx = (int)nx; op->st.ny = (int)ny; op->st.nz = (int)nz;
    op->st.n = n;
    op->st.D = D; op->st.Tx = Tx; op->st.Ty = Ty; op->st.Tz = dim == 3 ? Tz : nullptr;
    int rc = alloc_op(op);
    if (rc) { lc_op_destroy(op); return rc; }
    op->st.dinv = op->dinv;
    op->st.D32 = op->D32; op->st.Tx32 = op->Tx32; op->st.Ty32 = op->Ty32; op->st.Tz32 = op->Tz32;
    op->st.dinv32 = op->dinv32;
    op->st.sc = op->sc; op->st.sq = op->sq; op->st.Txh = op->Txh; op->st.Tyh = op->Tyh; op->st.Tzh = op->Tzh;
    op->st.dn32 = op->dn32; op->st.dexp = op->dexp;
    op->st.Txh32 = op->Txh32; op->st.Tyh32 = op->Tyh32; op->st.Tzh32 = op->Tzh32; op->st.sq32 = op->sq32;
    int *bad = reinterpret_cast<int *>(&op->ctrl->K);
    cudaError_t e = cudaMemset(bad, 0, sizeof(int));
    if (e == cudaSuccess) e = lc::launch_check_stencil(op->st, bad, 0);
    if (e == cudaSuccess)
        e = lc::launch_dinv_stencil(n, D, op->dinv, op->D32, Tx, Ty, op->st.Tz, op->Tx32, op->Ty32, op->Tz32,
                                    op->dinv32, 0);
    if (e == cudaSuccess)
        e = lc::launch_scaling(op->st, op->sc, op->sq, op->Txh, op->Tyh, op->Tzh, op->dn32, op->dexp, op->Txh32,
                               op->Tyh32, op->Tzh32, op->sq32, 0);
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "stencil set-up"); lc_op_destroy(op); return rc; }
    if (hbad) {
        lc_op_destroy(op);
        return fail(ctx, LC_ERR_INVALID_ARG, "stencil needs D > 0 and every interior face conductance > 0");
    }
    cudaMemset(op->ctrl, 0, sizeof(lc::Ctrl));
    *out = op;
    return LC_OK;
}

int lc_op_create_csr(lc_ctx *ctx, lc_op **out, int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                     const double *val) {
    if (!ctx || !out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n <= 0 || nnz < n) return fail(ctx, LC_ERR_INVALID_ARG, "need n > 0 and nnz >= n (diagonal present)");
    if (nnz >= (int64_t)INT32_MAX) return fail(ctx, LC_ERR_TOO_LARGE, "nnz = %lld does not fit int32", (long long)nnz);
    if (!rowptr || !col || !val) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    int32_t ends[2] = {0, 0};
    LC_CUDA(ctx, cudaMemcpy(&ends[0], rowptr, sizeof(int32_t), cudaMemcpyDeviceToHost));
    LC_CUDA(ctx, cudaMemcpy(&ends[1], rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (ends[0] != 0 || ends[1] != nnz) return fail(ctx, LC_ERR_INVALID_ARG, "rowptr[0] must be 0 and rowptr[n] = nnz");
    lc_op *op = new (std::nothrow) lc_op;
    if (!op) return LC_ERR_NO_MEMORY;
    op->ctx = ctx;
    ctx_ref(ctx);
    op->kind = 1;
    op->pcg_minblocks = 4;   // 64 registers, no spills: 32 warps per SM for the row-per-thread SpMV
    op->n = n;
    op->nnz = nnz;
    op->csr.n = n;
    op->csr.n_dev = nullptr;
    op->csr.rp = rowptr; op->csr.ci = col; op->csr.av = val;
    int rc = alloc_op(op);
    if (rc) { lc_op_destroy(op); return rc; }
    int *bad = reinterpret_cast<int *>(&op->ctrl->K);
    cudaError_t e = cudaMemset(bad, 0, sizeof(int));
    if (e == cudaSuccess) e = lc::launch_check_csr(n, rowptr, col, val, bad, 0);
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "CSR check"); lc_op_destroy(op); return rc; }
    if (hbad) {
        lc_op_destroy(op);
        return fail(ctx, LC_ERR_INVALID_ARG, "CSR rows must be sorted, unique, in range, with a positive diagonal");
    }
    cudaMemset(op->ctrl, 0, sizeof(lc::Ctrl));
    *out = op;
    return LC_OK;
}

int lc_op_destroy(lc_op *op) {
    if (!op) return LC_OK;
    if (op->ctx) cudaSetDevice(op->ctx->device);
    for (auto &ev : op->ev) if (ev) cudaEventDestroy(ev);
    for (auto &g : op->gslot) if (g.exec) cudaGraphExecDestroy(g.exec);
    if (op->cap) cudaStreamDestroy(op->cap);
    if (op->arena) cudaFree(op->arena);
    lc_ctx *ctx = op->ctx;
    delete op;
    ctx_unref(ctx);
    return LC_OK;
}

int lc_mark_residual(lc_ctx *ctx, const lc_op *op, const double *b, const double *x0, const lc_mark_params *p,
                     uint8_t *mask, double *r0_opt, int32_t *K_dev, double *tau_dev, void *stream) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!K_dev) return fail(ctx, LC_ERR_INVALID_ARG, "null K_dev");
    return mark_residual_impl(ctx, op, b, x0, p, mask, r0_opt, K_dev, tau_dev, (cudaStream_t)stream);
}

int lc_mark_gradient(lc_ctx *ctx, const lc_op *op, const double *x0, double alpha, int32_t layers, uint8_t *mask,
                     int32_t *K_dev, double *gmax_dev, void *stream) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!K_dev) return fail(ctx, LC_ERR_INVALID_ARG, "null K_dev");
    return mark_gradient_impl(ctx, op, x0, alpha, layers, mask, K_dev, gmax_dev, (cudaStream_t)stream);
}

int lc_extract(lc_ctx *ctx, const lc_op *op, const uint8_t *mask, const double *b, const double *x0,
               const lc_subsys *out, void *stream) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!out) return fail(ctx, LC_ERR_INVALID_ARG, "null subsystem");
    return extract_impl(ctx, op, mask, b, x0, *out, (cudaStream_t)stream);
}

int lc_pcg_solve(lc_ctx *ctx, const lc_op *op, const double *b, double *x, const lc_solve_params *p, lc_stats *stats,
                 void *stream) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!b || !x) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if ((rc = check_solve_params(ctx, p))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char key[sizeof(lc_params) + 4 * sizeof(void *) + 16];
    const size_t kl = call_key(key, op, b, x, p, stats != nullptr);
    rc = run_graphed(ctx, const_cast<lc_op *>(op), 0, key, kl, s, [&](cudaStream_t q, bool cap) -> int {
        if (stats) LC_CUDA(ctx, record(op->ev[0], q, cap));
        const int r = pcg_impl(ctx, op, b, x, p, op->ctrl, false, q);
        if (r) return r;
        if (stats) LC_CUDA(ctx, record(op->ev[1], q, cap));
        return LC_OK;
    });
    if (rc) return rc;
    if (!stats) return LC_OK;
    LC_CUDA(ctx, cudaStreamSynchronize(s));
    lc::Ctrl c;
    if ((rc = read_ctrl(ctx, op->ctrl, &c))) return rc;
    memset(stats, 0, sizeof *stats);
    stats->n = (int32_t)op->n;
    stats->it_global = c.iters;
    stats->restarts = c.restarts;
    stats->early_exit = c.early;
    stats->relres_tilde = c.relres0;
    stats->relres_final = c.relres;
    stats->t_global_ms = elapsed_ms(op->ev[0], op->ev[1]);
    stats->t_total_ms = stats->t_global_ms;
    stats->status = status_of(c);
    if (stats->status == LC_ERR_TIMEOUT) return fail(ctx, LC_ERR_TIMEOUT, "grid barrier timed out");
    return stats->status;
}

int lc_selftest_barrier_timeout(lc_ctx *ctx, lc_op *op, int32_t blocks, double limit_ms, int32_t *status_out) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!status_out || !(limit_ms > 0.0) || limit_ms > 2000.0)
        return fail(ctx, LC_ERR_INVALID_ARG, "limit_ms must be in (0, 2000]");
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, ctx->device);
    if (clk_khz <= 0) clk_khz = 2070000;
    const long long cycles = (long long)(limit_ms * (double)clk_khz);
    int *passed = reinterpret_cast<int *>(&op->ctrl->K);
    LC_CUDA(ctx, lc::launch_barrier_timeout_selftest(op->ctrl, passed, blocks, cycles, 0));
    LC_CUDA(ctx, cudaDeviceSynchronize());
    lc::Ctrl c;
    if ((rc = read_ctrl(ctx, op->ctrl, &c))) return rc;
    *status_out = c.K ? LC_OK : c.status;   // a block that got through would be a barrier bug
    LC_CUDA(ctx, cudaMemset(op->ctrl, 0, sizeof(lc::Ctrl)));
    return LC_OK;
}

int lc_op_dot(lc_ctx *ctx, const lc_op *op, const double *x, const double *y, double *out, void *stream) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!x || !y || !out) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    LC_CUDA(ctx, lc::launch_dot(op->n, x, y, out, op->pw.partials, (cudaStream_t)stream));
    return LC_OK;
}

static int check_gs(lc_ctx *ctx, const lc_op *op, int sweeps);

static int check_heat_bc(lc_ctx *ctx, const int32_t bc_type[4], const double bc_val[4], lc::HeatBc &bc) {
    if (!bc_type || !bc_val) return fail(ctx, LC_ERR_INVALID_ARG, "null boundary conditions");
    for (int f = 0; f < 4; ++f) {
        if (bc_type[f] != LC_BC_DIRICHLET && bc_type[f] != LC_BC_NEUMANN)
            return fail(ctx, LC_ERR_INVALID_ARG, "unknown boundary type %d", bc_type[f]);
        if (bc_type[f] == LC_BC_DIRICHLET && !std::isfinite(bc_val[f]))
            return fail(ctx, LC_ERR_INVALID_ARG, "Dirichlet values must be finite");
        bc.type[f] = bc_type[f];
        bc.val[f] = bc_val[f];
    }
    return LC_OK;
}

int lc_heat2d_assemble(lc_ctx *ctx, const int32_t shape[2], double h, double dt, const int32_t bc_type[4],
                       const double bc_val[4], const double *kappa, const double *Tn, double *D, double *Tx,
                       double *Ty, double *b, void *stream) {
    if (!ctx) return LC_ERR_INVALID_ARG;
    if (!shape || !kappa || !Tn || !D || !Tx || !Ty || !b) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if (shape[0] <= 0 || shape[1] <= 0) return fail(ctx, LC_ERR_INVALID_ARG, "shape must be positive");
    if ((int64_t)shape[0] * shape[1] >= (int64_t)INT32_MAX) return fail(ctx, LC_ERR_TOO_LARGE, "grid too large");
    if (!(h > 0.0) || !(dt > 0.0) || !std::isfinite(h) || !std::isfinite(dt))
        return fail(ctx, LC_ERR_INVALID_ARG, "h and dt must be positive and finite");
    lc::HeatBc bc;
    int rc = check_heat_bc(ctx, bc_type, bc_val, bc);
    if (rc) return rc;
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    LC_CUDA(ctx, lc::launch_heat_assemble(shape[0], shape[1], h, dt, bc, kappa, Tn, D, Tx, Ty, b,
                                          (cudaStream_t)stream));
    return LC_OK;
}

int lc_heat2d_step(lc_ctx *ctx, lc_op *op, const lc_heat2d_params *hp, const double *Tn, double *T, double *D,
                   double *Tx, double *Ty, double *b, double *work, lc_heat2d_stats *hs, void *stream) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!hp || !Tn || !T || !D || !Tx || !Ty || !b || !work || !hs)
        return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if (op->kind != 0 || op->st.dim != 2) return fail(ctx, LC_ERR_INVALID_ARG, "needs a 2D stencil operator");
    if (op->st.D != D || op->st.Tx != Tx || op->st.Ty != Ty)
        return fail(ctx, LC_ERR_INVALID_ARG, "D, Tx, Ty must be the arrays the operator was created on");
    if (!(hp->h > 0.0) || !(hp->dt > 0.0) || !std::isfinite(hp->h) || !std::isfinite(hp->dt) ||
        !std::isfinite(hp->p))
        return fail(ctx, LC_ERR_INVALID_ARG, "h, dt must be positive and p finite");
    if (hp->max_picard < 1 || !(hp->picard_tol >= 0.0)) return fail(ctx, LC_ERR_INVALID_ARG, "bad Picard limits");
    if (hp->method != 0 && hp->method != 1) return fail(ctx, LC_ERR_INVALID_ARG, "method must be 0 or 1");
    lc::HeatBc bc;
    if ((rc = check_heat_bc(ctx, hp->bc_type, hp->bc_val, bc))) return rc;
    if ((rc = check_solve_params(ctx, &hp->params.global))) return rc;
    if (hp->method == 1 && ((rc = check_solve_params(ctx, &hp->params.local)) ||
                            (rc = check_gs(ctx, op, hp->params.gs_sweeps))))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = op->n;
    double *kappa = work, *Tprev = work + n;
    double *part = op->pw.partials, *d2 = op->pw.partials + lc::kMaxGrid;
    memset(hs, 0, sizeof *hs);
    LC_CUDA(ctx, cudaEventRecord(op->ev[6], s));
    for (int it = 0; it < hp->max_picard; ++it) {
        LC_CUDA(ctx, lc::launch_heat_kappa(n, T, hp->p, kappa, s));
        LC_CUDA(ctx, lc::launch_heat_assemble(op->st.nx, op->st.ny, hp->h, hp->dt, bc, kappa, Tn, D, Tx, Ty, b, s));
        if ((rc = lc_op_refresh(op, stream))) return rc;
        LC_CUDA(ctx, cudaMemcpyAsync(Tprev, T, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        lc_stats st;
        rc = hp->method == 0 ? lc_pcg_solve(ctx, op, b, T, &hp->params.global, &st, stream)
                             : lc_solve_local_then_global(ctx, op, b, T, &hp->params, &st, stream);
        hs->status = rc;
        if (rc) return rc;
        hs->it_local += st.it_local;
        hs->it_global += st.it_global;
        hs->K_sum += st.K;
        hs->early_exits += st.early_exit;
        hs->t_solve_ms += st.t_total_ms;
        LC_CUDA(ctx, lc::launch_diff2(n, T, Tprev, part, d2, s));
        double h2 = 0.0;
        LC_CUDA(ctx, cudaMemcpyAsync(&h2, d2, sizeof(double), cudaMemcpyDeviceToHost, s));
        LC_CUDA(ctx, cudaStreamSynchronize(s));
        hs->picard_its = it + 1;
        hs->last_update = std::sqrt(h2);
        if (hs->last_update < hp->picard_tol) break;
    }
    LC_CUDA(ctx, cudaEventRecord(op->ev[7], s));
    LC_CUDA(ctx, cudaEventSynchronize(op->ev[7]));
    cudaEventElapsedTime(&hs->t_total_ms, op->ev[6], op->ev[7]);
    return LC_OK;
}

static constexpr int kMaxGsSweeps = 64;

static int check_gs(lc_ctx *ctx, const lc_op *op, int sweeps) {
    if (sweeps < 0 || sweeps > kMaxGsSweeps)
        return fail(ctx, LC_ERR_INVALID_ARG, "gs_sweeps must be 0..%d", kMaxGsSweeps);
    if (sweeps > 0 && op->kind != 0 && !op->colour)
        return fail(ctx, LC_ERR_UNSUPPORTED, "Gauss-Seidel on a CSR operator needs a colouring (lc_op_set_colouring)");
    return LC_OK;
}

static int gs_impl(lc_ctx *ctx, const lc_op *op, const double *b, double *x, int sweeps, cudaStream_t s) {
    if (sweeps <= 0 || op->n == 0) return LC_OK;
    if (op->kind == 0) LC_CUDA(ctx, lc::launch_gs_stencil(op->st, b, x, sweeps, s));
    else LC_CUDA(ctx, lc::launch_gs_csr(op->csr, op->colour, op->ncolours, b, x, sweeps, s));
    return LC_OK;
}

int lc_gs_smooth(lc_ctx *ctx, const lc_op *op, const double *b, double *x, int32_t sweeps, void *stream) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!b || !x) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if ((rc = check_gs(ctx, op, sweeps))) return rc;
    return gs_impl(ctx, op, b, x, sweeps, (cudaStream_t)stream);
}

int lc_op_set_colouring(lc_op *op, const uint8_t *colour, int32_t ncolours) {
    if (!op) return LC_ERR_INVALID_ARG;
    lc_ctx *ctx = op->ctx;
    if (op->kind == 0) return fail(ctx, LC_ERR_INVALID_ARG, "stencil operators use the red-black colouring");
    if (!colour) {
        op->colour = nullptr;
        op->ncolours = 0;
        return LC_OK;
    }
    if (ncolours < 1 || ncolours > 255) return fail(ctx, LC_ERR_INVALID_ARG, "ncolours must be 1..255");
    LC_CUDA(ctx, cudaSetDevice(ctx->device));
    int *bad = reinterpret_cast<int *>(&op->ctrl->K);
    LC_CUDA(ctx, cudaMemset(bad, 0, sizeof(int)));
    LC_CUDA(ctx, lc::launch_check_colouring(op->csr, colour, ncolours, bad, 0));
    int hbad = 0;
    LC_CUDA(ctx, cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost));
    if (hbad) return fail(ctx, LC_ERR_INVALID_ARG, "colouring out of range or two neighbours share a colour");
    op->colour = colour;
    op->ncolours = ncolours;
    return LC_OK;
}

int lc_solve_local_then_global(lc_ctx *ctx, const lc_op *op, const double *b, double *x, const lc_params *p,
                               lc_stats *stats, void *stream) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!b || !x || !p) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if ((rc = check_solve_params(ctx, &p->global)) || (rc = check_solve_params(ctx, &p->local))) return rc;
    if ((rc = check_gs(ctx, op, p->gs_sweeps))) return rc;
    if (p->mark_mode != LC_MARK_RESIDUAL && p->mark_mode != LC_MARK_GRADIENT)
        return fail(ctx, LC_ERR_INVALID_ARG, "unknown marking mode %d", p->mark_mode);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char key[sizeof(lc_params) + 4 * sizeof(void *) + 16];
    const size_t kl = call_key(key, op, b, x, p, stats != nullptr);
    rc = run_graphed(ctx, const_cast<lc_op *>(op), 1, key, kl, s, [&](cudaStream_t q, bool cap) -> int {
        int r;
        if (stats) LC_CUDA(ctx, record(op->ev[0], q, cap));
        // 1. local domain (Alg 2 or Alg 3)
        if (p->mark_mode == LC_MARK_RESIDUAL)
            r = mark_residual_impl(ctx, op, b, x, &p->mark, op->mask_own, nullptr, op->sub.K, nullptr, q);
        else
            r = mark_gradient_impl(ctx, op, x, p->alpha, p->grad_layers, op->mask_own, op->sub.K, nullptr, q);
        if (r) return r;
        if (stats) LC_CUDA(ctx, record(op->ev[1], q, cap));
        // 2. subsystem B x_B = b_B - E x_C (Eq. loc-equ)
        if ((r = extract_impl(ctx, op, op->mask_own, b, x, op->sub, q))) return r;
        if (stats) LC_CUDA(ctx, record(op->ev[2], q, cap));
        // 3. local solve from x0 restricted to the domain, in place in sub.xL0
        if ((r = pcg_impl(ctx, op, op->sub.rhs, op->sub.xL0, &p->local, op->ctrl_loc, true, q))) return r;
        // 4. x~ = x0 with the local solution scattered in (Eq. sol-assemble)
        LC_CUDA(ctx, lc::launch_assemble(op->sub.K, op->sub.l2g, op->sub.xL0, x, op->n, q));
        // 5. Gauss-Seidel smoothing of x~ over the whole system (step 7)
        if ((r = gs_impl(ctx, op, b, x, p->gs_sweeps, q))) return r;
        if (stats) LC_CUDA(ctx, record(op->ev[3], q, cap));
        // 6. convergence check of x~ and, if needed, the global solve from x~
        if ((r = pcg_impl(ctx, op, b, x, &p->global, op->ctrl, false, q))) return r;
        if (stats) LC_CUDA(ctx, record(op->ev[4], q, cap));
        return LC_OK;
    });
    if (rc) return rc;
    if (!stats) return LC_OK;
    LC_CUDA(ctx, cudaStreamSynchronize(s));
    lc::Ctrl cg, cl;
    if ((rc = read_ctrl(ctx, op->ctrl, &cg)) || (rc = read_ctrl(ctx, op->ctrl_loc, &cl))) return rc;
    memset(stats, 0, sizeof *stats);
    stats->n = (int32_t)op->n;
    stats->K = cg.K;
    stats->nnzB = cg.nnzB;
    stats->eta = op->n ? (double)cg.K / (double)op->n : 0.0;
    stats->tau = cg.tau;
    stats->it_local = cl.iters;
    stats->it_global = cg.iters;
    stats->early_exit = cg.early;
    stats->restarts = cg.restarts;
    stats->relres_tilde = cg.relres0;
    stats->relres_final = cg.relres;
    stats->t_mark_ms = elapsed_ms(op->ev[0], op->ev[1]);
    stats->t_extract_ms = elapsed_ms(op->ev[1], op->ev[2]);
    stats->t_local_ms = elapsed_ms(op->ev[2], op->ev[3]);
    stats->t_global_ms = elapsed_ms(op->ev[3], op->ev[4]);
    stats->t_total_ms = elapsed_ms(op->ev[0], op->ev[4]);
    int st = cl.status != LC_OK ? cl.status : (cl.converged == -1 && cg.K > 0 ? LC_ERR_BREAKDOWN : LC_OK);
    if (st == LC_OK) st = status_of(cg);
    stats->status = st;
    if (st == LC_ERR_TIMEOUT) return fail(ctx, LC_ERR_TIMEOUT, "grid barrier timed out");
    return st;
}

int lc_adjoint_grad(lc_ctx *ctx, lc_op *op, const double *k, double dt, const double *x, const double *gx,
                    double *lambda, double *dk, const lc_params *p, lc_stats *stats, void *stream) {
    int rc = check_common(ctx, op);
    if (rc) return rc;
    if (!k || !x || !gx || !lambda || !dk || !p) return fail(ctx, LC_ERR_INVALID_ARG, "null argument");
    if (op->kind != 0 || op->st.dim != 2)
        return fail(ctx, LC_ERR_INVALID_ARG, "the adjoint needs a 2D stencil operator of lc_assemble_diffusion_2d");
    const int32_t shape[2] = {op->st.nx, op->st.ny};
    // A(k) recomputed from k into the operator's own coefficient arrays (no
    // state of the forward solve is kept), then its derived data
    if ((rc = lc_assemble_diffusion_2d(ctx, shape, k, dt, const_cast<double *>(op->st.D),
                                       const_cast<double *>(op->st.Tx), const_cast<double *>(op->st.Ty), stream)))
        return rc;
    if ((rc = lc_op_refresh(op, stream))) return rc;
    // A lambda = dL/dx on the local-then-global path (A is symmetric)
    rc = lc_solve_local_then_global(ctx, op, gx, lambda, p, stats, stream);
    if (rc) return rc;
    return lc_adjoint_grad_k_2d(ctx, shape, k, x, lambda, dk, stream);
}

}  // extern "C"
