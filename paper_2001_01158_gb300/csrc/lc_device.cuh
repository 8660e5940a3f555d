// lc_device.cuh -- descriptors and device helpers shared by the lc kernels:
// operator descriptors, the control block, bit helpers, warp/block
// reductions and the bounded grid barrier.
//
// Nothing here is part of the public ABI (include/lc_api.h).  All kernels
// are written for sm_103a: 32-wide warps, 152 SMs, FP64 at roughly 1/12 of
// a DP op per HBM byte -- so every bit-exact kernel spends exactly the FP64
// operations its canonical order names and does abs/max/compare on integer
// bit patterns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lc_api.h"

namespace lc {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTreeChunk = 1024;                       // canonical sum-of-squares chunk
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;
constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr int kMaxExpRounds = 64;
constexpr int kMaxGrid = 4096;                          // persistent-kernel blocks (partials capacity)
constexpr int kPartialSlots = 16;                       // grid-reduction slots of kMaxGrid partials each

// ---------------------------------------------------------------- bounds-checked build
//
// Built with -DLC_CHECKED (a separate library, `build_library(checked=True)`),
// every index a kernel takes from data -- CSR column indices, the
// compaction's g2l / l2g maps -- is tested against its range before it is
// used.  A failing index is replaced by 0 (an element that exists) and the
// first failure's source line is recorded in the translation unit's check
// word; lc_checked_status() collects and clears the words of all units.  It
// stands in for a memory checker that this environment does not run; the
// ordinary build compiles LC_IDX to the bare index.
void register_check_word(unsigned (*take)(), const char *unit);
#ifdef LC_CHECKED
namespace {
__device__ unsigned g_check_word;
template <class I>
__device__ __forceinline__ I checked_index(I i, long long n, unsigned line) {
    if (!((long long)i >= 0 && (long long)i < n)) {
        atomicCAS(&g_check_word, 0u, line);
        return I(0);
    }
    return i;
}
unsigned take_check_word() {
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_check_word, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_check_word, &z, sizeof z) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
struct CheckWordRegistration {
    CheckWordRegistration() { register_check_word(&take_check_word, __BASE_FILE__); }
} check_word_registration;
}  // namespace
#define LC_IDX(i, n) ::lc::checked_index((i), (long long)(n), (unsigned)__LINE__)
#else
#define LC_IDX(i, n) (i)
#endif

// ---------------------------------------------------------------- descriptors

// Structured operator: the diagonal D and face conductances T (off-diagonal
// -T); dinv = 1/D precomputed at creation.  Cell i = x + nx*(y + ny*z).
struct Stencil {
    int dim;
    int nx, ny, nz;
    int64_t n;
    const double *D, *Tx, *Ty, *Tz;
    const double *dinv;
    // FP32 copies for the mixed-precision inner solve (fl32 of the above)
    const float *D32, *Tx32, *Ty32, *Tz32, *dinv32;
    // symmetric Jacobi scaling S = D^-1/2 (FP64 solve): S^-1 = D^1/2 and the
    // scaled face conductances T_f / sqrt(D_P D_N) of S A S (unit diagonal);
    // dn32 = fl32(D 2^-2h), h = floor(e/2), e the largest binary exponent of
    // D, stored biased (+1023) in *dexp
    const double *sc, *sq, *Txh, *Tyh, *Tzh;
    const float *dn32;
    const int *dexp;
    // the same scaling in FP32 for the mixed-precision inner solve: fl32 of
    // the scaled faces and of D^1/2 (weights of its true-residual norm)
    const float *Txh32, *Tyh32, *Tzh32, *sq32;
};

// CSR operator; rows ascending, diagonal present.  `n_dev`, if not null,
// holds the row count on the device (used for extracted subsystems whose
// size is only known on the device); otherwise `n` is the count.
struct Csr {
    int32_t n;
    const int32_t *n_dev;
    const int32_t *rp, *ci;
    const double *av;
    const float *av32;
};

// Device-resident control block of one operator (one per lc_op).
struct Ctrl {
    // grid barrier
    unsigned long long bar_count;   // arrivals since the launch started (zeroed before it)
    int32_t status;                 // first error a kernel raised (LC_OK if none)
    int32_t done;                   // local solve: 1 if the cluster kernel solved the system
    // marking
    unsigned long long maxabs_bits; // max |r| (or max g) as bits, NaN excluded
    double tau;
    int32_t K;
    int32_t nnzB;
    int32_t added[kMaxExpRounds];   // Alg 3: K0 of each round
    // Krylov
    int32_t iters;
    int32_t restarts;
    int32_t converged;              // 1 ok, 0 not converged, -1 breakdown
    int32_t early;                  // converged at set-up (x0 already met the criterion)
    double relres0;                 // relative residual of the starting iterate
    double relres;                  // final relative residual (true residual)
    double bnorm2;                  // ||b||^2
    // mixed-precision refinement
    int32_t outer;
    int32_t pad1;
    double scale;                   // ||r|| of the current outer residual
};

// ---------------------------------------------------------------- bit helpers

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & kAbsMask;
}
// |v| > t exactly as IEEE compares it, given tbits = abs_bits(t), t >= 0 or
// NaN: a NaN |v| never exceeds, nothing exceeds a NaN t or +inf.
__device__ __forceinline__ bool abs_gt(double v, unsigned long long tbits) {
    unsigned long long a = abs_bits(v);
    return a > tbits && a <= kInfBits && tbits <= kInfBits;
}
// bits of |v| for a max that ignores NaN (as `if (|v| > m) m = |v|` does)
__device__ __forceinline__ unsigned long long maxable_bits(double v) {
    unsigned long long a = abs_bits(v);
    return a <= kInfBits ? a : 0ull;
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_down_sync(kFull, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ int warp_isum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// Deterministic block sum of NV values per thread (result valid in thread 0).
// `sm` needs NV * 32 doubles.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[k * 32 + warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            T t = lane < nw ? sm[k * 32 + lane] : T(0);
            v[k] = warp_sum(t);
        }
    }
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sm[lane] : 0ull;
        v = warp_max(v);
    }
    return v;
}

__device__ __forceinline__ int block_isum(int v, int *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_isum(v);
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sm[lane] : 0;
        v = warp_isum(v);
    }
    return v;
}

// ---------------------------------------------------------------- grid barrier

// Spin limit of every grid-wide wait: ~2 s at 2 GHz, after which the block
// records LC_ERR_TIMEOUT in ctrl->status and returns false; the other blocks
// stop at their own next wait, bounded the same way, and kernels exit.  Co-residency of all
// blocks is guaranteed by the cooperative launch.
constexpr long long kBarrierTimeoutCycles = 4000000000ll;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Counting barrier: arrival k of a block (k = 0, 1, ...) takes the counter
// from somewhere in [k n, (k+1) n) and the barrier opens when it reaches
// (k+1) n, so the target follows from the value the arrival returns: one
// atomic per block and arrival, no generation word, no reset between
// barriers.  A block never sees the counter past its own target before it
// arrives (no block passes barrier k before all arrived).
// The arrival is a release add at GPU scope (it publishes the block's writes,
// ordered before it by the block barrier), the wait an acquire load: no
// separate fences.
__device__ __forceinline__ unsigned long long atom_add_release_u64(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ bool grid_sync(Ctrl *ctrl, unsigned int nblocks,
                                          long long limit_cycles = kBarrierTimeoutCycles) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long old = atom_add_release_u64(&ctrl->bar_count, 1ull);
        const unsigned long long target = (old / nblocks + 1) * nblocks;
        int ok = 1;
        if (old + 1 < target) {
            const long long t0 = clock64();
            while (ld_acquire_u64(&ctrl->bar_count) < target) {
                if (clock64() - t0 > limit_cycles) { ok = 0; break; }
            }
        }
        if (!ok) atomicCAS(&ctrl->status, LC_OK, LC_ERR_TIMEOUT);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Loads of data that other blocks of the same (persistent) kernel write:
// bypass L1, which is not coherent across SMs.
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// ---------------------------------------------------------------- grid reductions

struct NoPost {
    __device__ void operator()(double *) const {}
};

// The grid-wide part of a reduction whose block partials sit in slots
// `slot0..` (thread 0 wrote them): barrier, then warp 0 adds the block
// partials lane-strided and reduces them in a fixed order (identical in
// every block).  Thread 0 then runs post(t) on t[0..NV) = the totals, which
// may append ND derived scalars t[NV..NV+ND) (the CG step lengths): FP64
// divisions and tests run once per block instead of once per thread -- FP64
// issue is scarce.  Every thread reads the totals and derived values back.
// False if a wait timed out.
template <int NV, int ND, class Post>
__device__ __forceinline__ bool grid_tail(int slot0, double *part, double *red, Ctrl *ctrl, double (&out)[NV + ND],
                                          Post post) {
    if (!grid_sync(ctrl, gridDim.x)) return false;
    if (threadIdx.x < 32) {
        double acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += 32)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += ldcg(part + (size_t)(slot0 + k) * kMaxGrid + b);
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = warp_sum(acc[k]);
        if (threadIdx.x == 0) {
            double t[NV + ND];
#pragma unroll
            for (int k = 0; k < NV; ++k) t[k] = acc[k];
            post(t);
#pragma unroll
            for (int k = 0; k < NV + ND; ++k) red[96 + k] = t[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV + ND; ++k) out[k] = red[96 + k];
    __syncthreads();
    return true;
}

// Block sums of NV thread values into partial slots `slot0..`, then the
// grid-wide sums (grid_tail).
template <int NV, int ND = 0, typename T, class Post = NoPost>
__device__ __forceinline__ bool grid_sums(T (&v)[NV], int slot0, double *part, double *red, Ctrl *ctrl,
                                          double (&out)[NV + ND], Post post = Post()) {
    T tmp[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) tmp[k] = v[k];
    block_sum<NV, T>(tmp, reinterpret_cast<T *>(red));
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) part[(size_t)(slot0 + k) * kMaxGrid + blockIdx.x] = (double)tmp[k];
    return grid_tail<NV, ND>(slot0, part, red, ctrl, out, post);
}

// (ah, al) += (bh, bl) for FP32 pairs (Knuth's two-sum of the high parts).
__device__ __forceinline__ void pair_add(float &ah, float &al, float bh, float bl) {
    const float s = __fadd_rn(ah, bh);
    const float bv = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bv)), __fsub_rn(bh, bv));
    ah = s;
    al = __fadd_rn(al, __fadd_rn(bl, err));
}

// grid_sums with the block sums taken on FP32 pairs: thread value k is
// (h[k] + l[k]) 2^e[k]; warps and the block add pairs with FP32 two-sums
// (no FP64 instruction per thread), and thread 0 writes the block partial
// in FP64.  The grid-wide part is grid_tail's.
template <int NV, int ND = 0, class Post = NoPost>
__device__ __forceinline__ bool grid_sums_pair(const float (&h)[NV], const float (&l)[NV], const int (&e)[NV],
                                               int slot0, double *part, double *red, Ctrl *ctrl,
                                               double (&out)[NV + ND], Post post = Post()) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    float a[NV], b[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) { a[k] = h[k]; b[k] = l[k]; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float bh = __shfl_down_sync(kFull, a[k], o), bl = __shfl_down_sync(kFull, b[k], o);
            pair_add(a[k], b[k], bh, bl);
        }
    float *fs = reinterpret_cast<float *>(red);   // 2 NV x 32 floats
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) { fs[(2 * k) * 32 + warp] = a[k]; fs[(2 * k + 1) * 32 + warp] = b[k]; }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            a[k] = lane < nw ? fs[(2 * k) * 32 + lane] : 0.0f;
            b[k] = lane < nw ? fs[(2 * k + 1) * 32 + lane] : 0.0f;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const float bh = __shfl_down_sync(kFull, a[k], o), bl = __shfl_down_sync(kFull, b[k], o);
                pair_add(a[k], b[k], bh, bl);
            }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k)
                part[(size_t)(slot0 + k) * kMaxGrid + blockIdx.x] = ldexp((double)a[k] + (double)b[k], e[k]);
    }
    return grid_tail<NV, ND>(slot0, part, red, ctrl, out, post);
}

// A flag stored as a double by post(): tested with an integer compare.
__device__ __forceinline__ bool flag_set(double f) { return __double_as_longlong(f) != 0; }


}  // namespace lc
