// lc_pcgcsr.cu -- launch of the CSR Krylov solves (global CSR operators and
// the extracted local subsystems; FP64 and mixed precision); the kernels are
// in lc_pcg_impl.cuh.
#include "lc_pcg_impl.cuh"

namespace lc {

cudaError_t launch_pcg_csr(const Csr &op, const PcgArgs &a0, PcgWork &w, Ctrl *ctrl, int grid_hint, cudaStream_t s,
                           bool after_cluster) {
    // the row count may live on the device (extracted subsystem): the kernels
    // are sized for the capacity op.n and read the actual count themselves
    const int64_t units = (op.n + kPcgThreads - 1) / kPcgThreads;
    // 768-thread blocks only for extracted subsystems: small systems gain
    // from fewer blocks per reduction (2048^2 Alg 1 local solve: 13.6 ->
    // 11.7 us per iteration), large gather-bound ones lose warps per SM
    PcgArgs a = a0;
    a.big = a0.big && op.n_dev != nullptr;
    csr_dinv_kernel<double><<<152 * 4, 256, 0, s>>>(op, op.av, w.dinv);
    note_launches(1);
    Vecs<double> VD = vecs64(a, w, w.dinv);
    OpCsr<double> od{op, op.av, op.n};
    if (after_cluster) {
        od.done = &ctrl->done;
        return launch_pcg(od, units, VD, w.partials, a, ctrl, grid_hint, a.minblocks, s, false);
    }
    // a global system stores p once per row (OpCsr SP); an extracted
    // subsystem, latency-bound, recomputes it at the columns (no extra barrier)
    const bool sp = a.store_p && op.n_dev == nullptr;
    if (a.precision != LC_PREC_MIXED) {
        if (sp) {
            OpCsr<double, true> os{op, op.av, op.n};
            os.bar = ctrl;
            return launch_pcg(os, units, VD, w.partials, a, ctrl, grid_hint, a.minblocks, s);
        }
        return launch_pcg(od, units, VD, w.partials, a, ctrl, grid_hint, a.minblocks, s);
    }
    VD.z = nullptr;
    const float *av32 = op.av32;
    if (!av32) {   // per-solve FP32 copy of the values into the workspace
        csr_to_f32_kernel<<<152 * 8, 256, 0, s>>>(op, w.val32);
        note_launches(1);
        av32 = w.val32;
    }
    csr_dinv_kernel<float><<<152 * 4, 256, 0, s>>>(op, av32, w.dinv32);
    note_launches(1);
    Vecs<float> VF = vecs32(w, w.dinv32);
    if (sp) {
        OpCsr<float, true> ofs{op, av32, op.n};
        ofs.bar = ctrl;
        return launch_ir(od, ofs, units, VD, VF, w.partials, a, ctrl, grid_hint, a.minblocks, s);
    }
    OpCsr<float> of{op, av32, op.n};
    return launch_ir(od, of, units, VD, VF, w.partials, a, ctrl, grid_hint, a.minblocks, s);
}

}  // namespace lc
