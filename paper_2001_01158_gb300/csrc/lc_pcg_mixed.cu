// lc_pcg_mixed.cu -- launch of the 2D mixed-precision solves (FP32 inner
// Jacobi-CG inside FP64 iterative refinement, one persistent launch); the
// kernels are in lc_pcg_impl.cuh.
#include "lc_pcg_impl.cuh"

namespace lc {

cudaError_t launch_ir_stencil2d(const Stencil &op, const PcgArgs &a, PcgWork &w, Ctrl *ctrl, int grid_hint,
                                cudaStream_t s) {
    Vecs<double> VD = vecs64(a, w, op.dinv);
    VD.z = nullptr;   // the refinement residual needs no z
    Vecs<float> VF = vecs32(w, op.dinv32);
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    const bool vec = op.nx % 2 == 0 && al16(op.D) && al16(op.Tx) && al16(op.Ty);
    const int wpb = kPcgThreads / 32;
    if (vec) {
        const int64_t units = ((int64_t)((op.nx + 63) / 64) * op.ny + 4 * wpb - 1) / (4 * wpb);
        Op2DW<double, 2> od{op, coef64(op)};
        if (op.nx % 4 == 0 && a.scaled && op.Txh32) {   // the inner solve on the scaled system
            Op2DW<float, 4, true> of{op, Coef<float>{op.D32, op.Txh32, op.Tyh32, nullptr}, op.sc, op.sq, op.sq32,
                                     nullptr};
            Vecs<float> VS = VF;
            VS.z = VF.r;
            VS.dinv = nullptr;
            return launch_ir(od, of, units, VD, VS, w.partials, a, ctrl, grid_hint, a.minblocks, s);
        }
        if (op.nx % 4 == 0) {   // FP32 copies are the library's own, 256-byte aligned: float4 lanes
            Op2DW<float, 4> of{op, coef32(op)};
            return launch_ir(od, of, units, VD, VF, w.partials, a, ctrl, grid_hint, a.minblocks, s);
        }
        Op2DW<float, 2> of{op, coef32(op)};
        return launch_ir(od, of, units, VD, VF, w.partials, a, ctrl, grid_hint, a.minblocks, s);
    }
    const int64_t units = ((int64_t)((op.nx + 31) / 32) * op.ny + 4 * wpb - 1) / (4 * wpb);
    Op2DW<double, 1> od{op, coef64(op)};
    Op2DW<float, 1> of{op, coef32(op)};
    return launch_ir(od, of, units, VD, VF, w.partials, a, ctrl, grid_hint, a.minblocks, s);
}

}  // namespace lc
