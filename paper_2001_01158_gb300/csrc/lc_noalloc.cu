// lc_noalloc.cu -- residual marking that allocates no device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's memory pool or under a strict memory budget, or a host that
// must not allocate after start-up.  For them
// lc_mark_residual_stencil_noalloc computes the same local domain as
// lc_mark_residual on a structured operator, but its scratch memory (the
// control block, the sum-of-squares tree partials and the second mask
// buffer of multi-pass expansion) lives in the fixed file-scope device array
// below instead of an operator workspace.  Every device that loads the
// library holds this array until the process exits.
#include "lc_internal.cuh"

namespace {

constexpr int64_t kMaxCells = LC_NOALLOC_MAX_CELLS;
constexpr size_t kTreeSlots = (size_t)((kMaxCells + lc::kTreeChunk - 1) / lc::kTreeChunk) + 2;
constexpr size_t kCtrlBytes = (sizeof(lc::Ctrl) + 255) / 256 * 256;
constexpr size_t kTreeBytes = (kTreeSlots * sizeof(double) + 255) / 256 * 256;
constexpr size_t kOffTreeA = kCtrlBytes;
constexpr size_t kOffTreeB = kOffTreeA + kTreeBytes;
constexpr size_t kOffMask = kOffTreeB + kTreeBytes;
constexpr size_t kScratchBytes = kOffMask + (size_t)kMaxCells;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array for the context current on the calling
// thread.  It is looked up on every call (cudaGetSymbolAddress is a host-side
// table lookup once the module is loaded) rather than cached: if the device's
// context is torn down and created again (cudaDeviceReset, or a framework
// that resets the device), the module is loaded anew and the array may sit at
// another address, which a cached pointer would not follow.
int scratch_address(unsigned char **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return LC_ERR_CUDA;
    }
    *out = static_cast<unsigned char *>(p);
    return LC_OK;
}

}  // namespace

extern "C" int lc_mark_residual_stencil_noalloc(int32_t dim, const int32_t shape[3], const double *D,
                                                const double *Tx, const double *Ty, const double *Tz,
                                                const double *b, const double *x0, const lc_mark_params *p,
                                                uint8_t *mask, double *r0, int32_t *K_dev, double *tau_dev,
                                                void *stream) {
    // argument checks come first and touch no GPU
    if (dim != 2 && dim != 3) return LC_ERR_INVALID_ARG;
    if (!shape || !D || !Tx || !Ty || (dim == 3 && !Tz) || !b || !x0 || !p || !mask || !r0 || !K_dev)
        return LC_ERR_INVALID_ARG;
    const int64_t nx = shape[0], ny = shape[1], nz = dim == 3 ? shape[2] : 1;
    if (nx <= 0 || ny <= 0 || nz <= 0) return LC_ERR_INVALID_ARG;
    if (nx * ny * nz > kMaxCells) return LC_ERR_TOO_LARGE;
    if (p->thr_mode != LC_THR_EPS_NORMB && p->thr_mode != LC_THR_REL_MAX) return LC_ERR_INVALID_ARG;
    if (!(p->thr_param >= 0.0) || p->thr_param > 1.7976931348623157e308) return LC_ERR_INVALID_ARG;
    if (p->exp_mode < LC_EXP_NONE || p->exp_mode > LC_EXP_PAPER) return LC_ERR_INVALID_ARG;
    if (p->exp_rounds < 0 || p->exp_rounds > lc::kMaxExpRounds) return LC_ERR_INVALID_ARG;

    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    lc::Ctrl *ctrl = reinterpret_cast<lc::Ctrl *>(base);
    double *tree_a = reinterpret_cast<double *>(base + kOffTreeA);
    double *tree_b = reinterpret_cast<double *>(base + kOffTreeB);
    uint8_t *tmp = base + kOffMask;

    lc::Stencil st{};
    st.dim = dim;
    st.nx = (int)nx; st.ny = (int)ny; st.nz = (int)nz;
    st.n = nx * ny * nz;
    st.D = D; st.Tx = Tx; st.Ty = Ty; st.Tz = dim == 3 ? Tz : nullptr;

    cudaStream_t s = (cudaStream_t)stream;
    const double param = p->thr_param == 0.0 ? 0.0 : p->thr_param;
    const int tree = p->thr_mode == LC_THR_EPS_NORMB;
#define NA_CUDA(call) do { if ((call) != cudaSuccess) { cudaGetLastError(); return LC_ERR_CUDA; } } while (0)
    // the control block starts at zero for every call (max, counts, tau)
    NA_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(lc::Ctrl), s));
    NA_CUDA(lc::launch_residual_stencil(st, b, x0, r0, tree, tree_a, ctrl, s));
    if (tree) {
        const int64_t nchunks = (st.n + lc::kTreeChunk - 1) / lc::kTreeChunk;
        NA_CUDA(lc::launch_tree_finish(tree_a, tree_b, nchunks, st.n, param, ctrl, tau_dev, s));
    } else {
        NA_CUDA(lc::launch_tau_relmax(param, ctrl, tau_dev, s));
    }
    const int rounds = p->exp_rounds;
    if (p->exp_mode == LC_EXP_DILATE && rounds > 0) {
        const int lmax = lc::max_layers_per_pass(dim);
        const int first = rounds < lmax ? rounds : lmax;
        const int rest = rounds - first;
        const int passes = 1 + (rest + lmax - 1) / lmax;
        uint8_t *cur = ((passes - 1) % 2 == 0) ? mask : tmp;
        NA_CUDA(lc::launch_threshold_dilate_stencil(st, r0, first, cur, ctrl, s));
        for (int left = rest; left > 0;) {
            const int l = left < lmax ? left : lmax;
            uint8_t *nxt = cur == mask ? tmp : mask;
            NA_CUDA(lc::launch_dilate_stencil_pass(st, l, cur, nxt, s));
            cur = nxt;
            left -= l;
        }
    } else if (p->exp_mode == LC_EXP_PAPER && rounds > 0) {
        uint8_t *cur = (rounds % 2 == 0) ? mask : tmp;
        NA_CUDA(lc::launch_threshold_dilate_stencil(st, r0, 0, cur, ctrl, s));
        for (int m = 0; m < rounds; ++m) {
            uint8_t *nxt = cur == mask ? tmp : mask;
            NA_CUDA(lc::launch_expand_paper_stencil(st, r0, x0, m, cur, nxt, ctrl, s));
            cur = nxt;
        }
    } else {
        NA_CUDA(lc::launch_threshold_dilate_stencil(st, r0, 0, mask, ctrl, s));
    }
    NA_CUDA(cudaMemsetAsync(&ctrl->K, 0, sizeof(int32_t), s));
    NA_CUDA(lc::launch_count_mask(st.n, mask, ctrl, K_dev, s));
#undef NA_CUDA
    return LC_OK;
}
