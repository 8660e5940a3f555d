// lc_pcg.cu -- launch of the 2D FP64 Krylov solves (the scaled four-cells-
// per-lane kernel that dominates the Alg 1 workload, and its variants), the
// dispatch to the 3D, mixed-precision and CSR launchers, and the operator
// set-up kernels (1/D, FP32 copies, the symmetric scaling, checks).  The
// kernels themselves are in lc_pcg_impl.cuh.
#include "lc_pcg_impl.cuh"

namespace lc {

cudaError_t launch_pcg_stencil(const Stencil &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                               cudaStream_t s) {
    if (op.dim == 3) return launch_pcg_stencil3d(op, a, w, ctrl, grid_hint, s);
    if (a.precision == LC_PREC_MIXED) return launch_ir_stencil2d(op, a, w, ctrl, grid_hint, s);
    Vecs<double> VD = vecs64(a, w, op.dinv);
    // two cells per lane (paired loads) when every row starts 16-byte aligned
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    const bool vec = op.nx % 2 == 0 && al16(op.D) && al16(op.Tx) && al16(op.Ty);
    const int wpb = kPcgThreads / 32;
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // blocks for strips of `width` columns: 4 rows per warp so the recomputed
    // halo rows stay a small overhead -- unless that leaves SMs idle (small
    // grids: 99 x 99 filled 5 SMs, 22 us per iteration), then 2 or 1 rows
    const auto units_for = [&](int width) {
        const int64_t rows = (int64_t)((op.nx + width - 1) / width) * op.ny;
        for (int r = 4;; r /= 2) {
            const int64_t u = (rows + (int64_t)r * wpb - 1) / ((int64_t)r * wpb);
            if (r == 1 || u >= sms) return u;
        }
    };
    if (vec) {
        const int64_t units = units_for(64);
        if (a.scaled && op.sc && a.wide && op.nx % 4 == 0) {
            // four cells per lane: half the strip-end halos and segment starts
            const int64_t units4 = units_for(128);
            const Coef<double> ch{op.D, op.Txh, op.Tyh, nullptr};
            Vecs<double> VS = VD;
            VS.x = w.z;
            VS.z = w.r;
            VS.dinv = nullptr;
            VS.xu = a.x;
            if (a.pairdot && a.lazyx) {   // and the x update riding on the next phase A
                Op2DW<double, 4, true, true, true> o3{op, ch, op.sc, op.sq, op.dn32, op.dexp};
                return launch_pcg(o3, units4, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
            }
            if (a.pairdot) {   // dot products and block sums on FP32 pairs
                Op2DW<double, 4, true, true> o2{op, ch, op.sc, op.sq, op.dn32, op.dexp};
                return launch_pcg(o2, units4, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
            }
            Op2DW<double, 4, true> os{op, ch, op.sc, op.sq, op.dn32, op.dexp};
            return launch_pcg(os, units4, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
        }
        if (a.scaled && op.sc) {
            // the symmetrically scaled system: x^ in the z workspace, z = r^
            Op2DW<double, 2, true> os{op, Coef<double>{op.D, op.Txh, op.Tyh, nullptr}, op.sc, op.sq, op.dn32,
                                      op.dexp};
            Vecs<double> VS = VD;
            VS.x = w.z;
            VS.z = w.r;
            VS.dinv = nullptr;
            VS.xu = a.x;
            return launch_pcg(os, units, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
        }
        Op2DW<double, 2> od{op, coef64(op)};
        return launch_pcg(od, units, VD, w.partials, a, ctrl, grid_hint, a.minblocks, s);
    }
    const int64_t units = units_for(32);
    if (a.scaled && op.sc) {   // odd widths: the scaled system one cell per lane
        Op2DW<double, 1, true> os{op, Coef<double>{op.D, op.Txh, op.Tyh, nullptr}, op.sc, op.sq, op.dn32, op.dexp};
        Vecs<double> VS = VD;
        VS.x = w.z;
        VS.z = w.r;
        VS.dinv = nullptr;
        VS.xu = a.x;
        return launch_pcg(os, units, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
    }
    Op2DW<double, 1> od{op, coef64(op)};
    return launch_pcg(od, units, VD, w.partials, a, ctrl, grid_hint, a.minblocks, s);
}

cudaError_t launch_dinv_stencil(int64_t n, const double *D, double *dinv, float *D32, const double *Tx,
                                const double *Ty, const double *Tz, float *Tx32, float *Ty32, float *Tz32,
                                float *dinv32, cudaStream_t s) {
    dinv_stencil_kernel<<<152 * 8, 256, 0, s>>>(n, D, dinv, D32, Tx, Ty, Tz, Tx32, Ty32, Tz32, dinv32);
    note_launches(1);
    return cudaGetLastError();
}

namespace {
__global__ void max_exponent_kernel(int64_t n, const double *__restrict__ D, int *dexp) {
    int m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (int)((__double_as_longlong(D[i]) >> 52) & 0x7ff));
    m = __reduce_max_sync(0xffffffffu, (unsigned)m);
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(dexp, m);
}

__global__ void scaling_kernel(Stencil st, double *sc, double *sq, double *Txh, double *Tyh, double *Tzh,
                               float *dn32, const int *dexp, float *Txh32, float *Tyh32, float *Tzh32, float *sq32) {
    const int64_t n = st.n, sxy = (int64_t)st.nx * st.ny;
    const int h = (*dexp - 1023) >> 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % st.nx), y = (int)((i / st.nx) % st.ny), z = (int)(i / sxy);
        const double r = sqrt(st.D[i]);
        const double s = 1.0 / r;
        sc[i] = s;
        sq[i] = r;
        const double tx = x + 1 < st.nx ? st.Tx[i] * s * (1.0 / sqrt(st.D[i + 1])) : 0.0;
        const double ty = y + 1 < st.ny ? st.Ty[i] * s * (1.0 / sqrt(st.D[i + st.nx])) : 0.0;
        Txh[i] = tx;
        Tyh[i] = ty;
        Txh32[i] = (float)tx;
        Tyh32[i] = (float)ty;
        if (st.dim == 3) {
            const double tz = z + 1 < st.nz ? st.Tz[i] * s * (1.0 / sqrt(st.D[i + sxy])) : 0.0;
            Tzh[i] = tz;
            Tzh32[i] = (float)tz;
        }
        dn32[i] = (float)ldexp(st.D[i], -2 * h);
        sq32[i] = (float)r;
    }
}
}  // namespace

cudaError_t launch_scaling(const Stencil &st, double *sc, double *sq, double *Txh, double *Tyh, double *Tzh,
                           float *dn32, int *dexp, float *Txh32, float *Tyh32, float *Tzh32, float *sq32,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(dexp, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    max_exponent_kernel<<<152 * 4, 256, 0, s>>>(st.n, st.D, dexp);
    scaling_kernel<<<152 * 8, 256, 0, s>>>(st, sc, sq, Txh, Tyh, Tzh, dn32, dexp, Txh32, Tyh32, Tzh32, sq32);
    note_launches(2);
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
