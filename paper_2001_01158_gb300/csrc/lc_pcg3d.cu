// lc_pcg3d.cu -- launch of the 3D Krylov solves (FP64 on the scaled system
// and its variants, mixed precision); the kernels are in lc_pcg_impl.cuh.
#include "lc_pcg_impl.cuh"

namespace lc {

cudaError_t launch_pcg_stencil3d(const Stencil &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                                 cudaStream_t s) {
    const bool mixed = a.precision == LC_PREC_MIXED;
    Vecs<double> VD = vecs64(a, w, op.dinv);
    if (mixed) VD.z = nullptr;   // the refinement residual needs no z
    Vecs<float> VF = vecs32(w, op.dinv32);
    const int64_t units = (int64_t)((op.nx + kTileX - 1) / kTileX) * ((op.ny + kTileY - 1) / kTileY) *
                          ((op.nz + kTileZ - 1) / kTileZ);
    Op3D<double> od{op, coef64(op)};
    if (!mixed && a.scaled && op.sc) {   // the symmetrically scaled system (as in 2D)
        Op3D<double, true> os{op, Coef<double>{op.D, op.Txh, op.Tyh, op.Tzh}, op.sc, op.sq, op.dn32, op.dexp};
        Vecs<double> VS = VD;
        VS.x = w.z;
        VS.z = w.r;
        VS.dinv = nullptr;
        VS.xu = a.x;
        if (a.pairdot && a.lazyx) {
            Op3D<double, true, true, true> o3{op, os.c, op.sc, op.sq, op.dn32, op.dexp};
            return launch_pcg(o3, units, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
        }
        if (a.pairdot) {
            Op3D<double, true, true> o2{op, os.c, op.sc, op.sq, op.dn32, op.dexp};
            return launch_pcg(o2, units, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
        }
        return launch_pcg(os, units, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
    }
    if (!mixed) return launch_pcg(od, units, VD, w.partials, a, ctrl, grid_hint, a.minblocks, s);
    if (a.scaled && op.Txh32) {
        Op3D<float, true> of{op, Coef<float>{op.D32, op.Txh32, op.Tyh32, op.Tzh32}, op.sc, op.sq, op.sq32,
                             nullptr};
        Vecs<float> VS = VF;
        VS.z = VF.r;
        VS.dinv = nullptr;
        return launch_ir(od, of, units, VD, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
    }
    Op3D<float> of{op, coef32(op)};
    return launch_ir(od, of, units, VD, VF, w.partials, a, ctrl, grid_hint, a.minblocks, s);
}

}  // namespace lc
