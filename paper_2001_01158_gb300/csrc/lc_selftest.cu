// lc_selftest.cu -- self-test of the bounded grid-wide wait: a cooperative
// launch whose barrier expects one arrival more than there are blocks, so
// the wait can only end by its limit.  Every block gives up after
// `limit_cycles`, records LC_ERR_TIMEOUT in the control block and returns;
// nothing faults, traps or hangs, and the context stays usable.
#include "lc_internal.cuh"

namespace lc {

namespace {

__global__ void barrier_timeout_kernel(Ctrl *ctrl, long long limit_cycles, int *passed) {
    // gridDim.x + 1 arrivals expected: the last one never comes
    const bool ok = grid_sync(ctrl, gridDim.x + 1, limit_cycles);
    if (threadIdx.x == 0 && ok) atomicAdd(passed, 1);
}

__global__ void reset_selftest_kernel(Ctrl *ctrl, int *passed) {
    ctrl->bar_count = 0;
    ctrl->status = LC_OK;
    *passed = 0;
}

}  // namespace

cudaError_t launch_barrier_timeout_selftest(Ctrl *ctrl, int *passed, int blocks, long long limit_cycles,
                                            cudaStream_t s) {
    reset_selftest_kernel<<<1, 1, 0, s>>>(ctrl, passed);
    int lim_blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lim_blocks, barrier_timeout_kernel, 128, 0);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks < 1) blocks = 1;
    if (blocks > lim_blocks * sms) blocks = lim_blocks * sms;
    Ctrl *c = ctrl;
    long long lim = limit_cycles;
    int *p = passed;
    void *args[] = {&c, &lim, &p};
    note_launches(2);
    return cudaLaunchCooperativeKernel((const void *)barrier_timeout_kernel, dim3(blocks), dim3(128), args, 0, s);
}

}  // namespace lc
