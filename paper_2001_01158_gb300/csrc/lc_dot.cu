// lc_dot.cu -- reproducible FP64 dot product: every product x_i y_i (one
// FP64 rounding) is converted to a 128-bit integer relative to the largest
// product's exponent, the integers are summed exactly (in any order: the
// result does not depend on the launch configuration), and the total is
// rounded once to a double.
#include "lc_internal.cuh"

namespace lc {

namespace {

// Exact, order-independent sums.  A double v = (-1)^s M 2^(e-1075) (e its
// biased exponent, M its 53-bit significand; subnormals e = 1) is
// written relative to a reference exponent E >= e as the 128-bit integer
//     F = M 2^(52 - (E - e))       exact while E - e <= 52, rounded beyond,
// so every term within 2^-52 of the largest is kept exactly and the integer
// sums are exact and independent of the order of addition (bits 105..126 are
// headroom for 2^21 terms; fewer fraction bits FB leave more).
typedef __int128 lc_i128;
typedef unsigned __int128 lc_u128;

constexpr int kFxBad = 1 << 16;   // exponent-word flag: a term was NaN or infinite

struct FxTerm {
    unsigned long long m;
    int e;
    bool neg, bad;
};

__device__ __forceinline__ FxTerm fx_split(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    FxTerm t;
    t.neg = (b >> 63) != 0;
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long frac = b & 0xfffffffffffffull;
    t.bad = e == 0x7ff;
    if (t.bad) { t.m = 0; t.e = 0; }
    else if (e == 0) { t.m = frac; t.e = frac ? 1 : 0; }
    else { t.m = frac | (1ull << 52); t.e = e; }
    return t;
}

// arithmetic right shift by k >= 0, rounding half away from zero in magnitude
__device__ __forceinline__ lc_i128 fx_shr(lc_i128 x, int k) {
    if (k <= 0) return x;
    if (k >= 126) return 0;
    const bool neg = x < 0;
    lc_u128 m = neg ? (lc_u128)(-x) : (lc_u128)x;
    m = (m + ((lc_u128)1 << (k - 1))) >> k;
    return neg ? -(lc_i128)m : (lc_i128)m;
}

// t relative to E >= t.e with FB fraction bits: M 2^(FB - (E - e)), exact
// while E - e <= FB, rounded to nearest beyond (the result scale is
// 2^(E - 1075 - FB))
template <int FB = 52>
__device__ __forceinline__ lc_i128 fx_scale(const FxTerm &t, int E) {
    if (t.m == 0) return 0;
    const int sh = E - t.e;
    lc_i128 r;
    if (sh <= FB) {
        r = (lc_i128)t.m << (FB - sh);
    } else {
        const int rs = sh - FB;
        if (rs > 53) return 0;
        r = (lc_i128)((t.m + (1ull << (rs - 1))) >> rs);
    }
    return t.neg ? -r : r;
}

__device__ __forceinline__ lc_i128 fx_shfl_down(lc_i128 v, int o) {
    unsigned long long lo = (unsigned long long)v;
    long long hi = (long long)(v >> 64);
    lo = __shfl_down_sync(kFull, lo, o);
    hi = __shfl_down_sync(kFull, hi, o);
    return (lc_i128)(((lc_u128)(unsigned long long)hi << 64) | (lc_u128)lo);
}

// (S, E) -> the double nearest S 2^(E - 1075 - FB) (ties to even); NaN if bad
template <int FB = 52>
__device__ __forceinline__ double fx_to_double(lc_i128 S, int E, bool bad) {
    if (bad) return __longlong_as_double(0x7ff8000000000000ll);
    if (S == 0) return 0.0;
    const bool neg = S < 0;
    const lc_u128 m = neg ? (lc_u128)(-S) : (lc_u128)S;
    const unsigned long long hi = (unsigned long long)(m >> 64), lo = (unsigned long long)m;
    const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    unsigned long long top;
    if (msb >= 63) {
        const int sh = msb - 63;
        top = (unsigned long long)(m >> sh);
        if (sh && (m & (((lc_u128)1 << sh) - 1))) top |= 1ull;   // sticky bit below the 64 kept
    } else {
        top = lo << (63 - msb);
    }
    const double d = ldexp(__ull2double_rn(top), msb - 63 + E - 1075 - FB);
    return neg ? -d : d;
}

constexpr int kDotFB = 40;   // fraction bits: 2^33 terms of headroom
constexpr int kDotThreads = 256;

__global__ void dot_maxexp_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ y, int *emax) {
    unsigned m = 0, bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const FxTerm t = fx_split(x[i] * y[i]);
        m = max(m, (unsigned)t.e);
        bad |= t.bad ? (unsigned)kFxBad : 0u;
    }
    m = __reduce_max_sync(kFull, m);
    bad = __reduce_or_sync(kFull, bad);
    if ((threadIdx.x & 31) == 0) {
        if (m) atomicMax(emax, (int)m);
        if (bad) atomicOr(emax, kFxBad);
    }
}

__global__ void dot_partial_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                                   const int *emax, unsigned long long *part) {
    __shared__ lc_i128 ws[32];
    const int E = *emax & ~kFxBad;
    lc_i128 acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += fx_scale<kDotFB>(fx_split(x[i] * y[i]), E);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += fx_shfl_down(acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        lc_i128 v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : (lc_i128)0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += fx_shfl_down(v, o);
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = (unsigned long long)v;
            part[2 * blockIdx.x + 1] = (unsigned long long)(v >> 64);
        }
    }
}

__global__ void dot_final_kernel(int nparts, const unsigned long long *part, const int *emax, double *out) {
    lc_i128 acc = 0;
    for (int b = threadIdx.x; b < nparts; b += 32)
        acc += (lc_i128)(((lc_u128)part[2 * b + 1] << 64) | (lc_u128)part[2 * b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += fx_shfl_down(acc, o);
    if (threadIdx.x == 0) {
        const int e = *emax;
        *out = fx_to_double<kDotFB>(acc, e & ~kFxBad, (e & kFxBad) != 0);
    }
}

}  // namespace

cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *out, double *scratch, cudaStream_t s) {
    int *emax = reinterpret_cast<int *>(scratch);
    unsigned long long *part = reinterpret_cast<unsigned long long *>(scratch) + 2;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + kDotThreads - 1) / kDotThreads, 152 * 4));
    cudaError_t e = cudaMemsetAsync(emax, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    dot_maxexp_kernel<<<grid, kDotThreads, 0, s>>>(n, x, y, emax);
    dot_partial_kernel<<<grid, kDotThreads, 0, s>>>(n, x, y, emax, part);
    dot_final_kernel<<<1, 32, 0, s>>>(grid, part, emax, out);
    note_launches(3);
    return cudaGetLastError();
}

}  // namespace lc
