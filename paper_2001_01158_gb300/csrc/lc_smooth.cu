// lc_smooth.cu -- Gauss-Seidel smoothing of x~ (Alg 1, step 7) over the whole
// system A x = b.
//
// Multicolour Gauss-Seidel: the points of one colour are updated together,
// colour after colour, each from the newest values of its neighbours.  No
// two neighbours share a colour, so every point of a colour reads only
// points of other colours and the result does not depend on the order
// inside a colour: the GPU updates a colour in parallel and matches the
// serial sweep bit for bit.  Per point, in the canonical order
//     s = b_i; for j ascending, j != i: s = fma(-a_ij, x_j, s); x_i = s / a_ii.
// Stencil operators use the red-black colouring (x + y + z) mod 2 of the
// grid; CSR operators use a colouring the caller supplies.
#include "lc_internal.cuh"

namespace lc {

namespace {

// One colour of a stencil sweep.  Thread item p covers the pair of cells
// (2k, 2k+1) of a row and updates the one of colour c.
__global__ void gs_stencil_kernel(Stencil s, const double *__restrict__ b, double *x, int c) {
    const int half = (s.nx + 1) >> 1;
    const int64_t items = (int64_t)half * s.ny * s.nz;
    const int64_t sxy = (int64_t)s.nx * s.ny;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < items;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(p % half);
        const int64_t row = p / half;
        const int y = (int)(row % s.ny), z = (int)(row / s.ny);
        const int xx = 2 * k + ((y + z + c) & 1);
        if (xx >= s.nx) continue;
        const int64_t i = (int64_t)z * sxy + (int64_t)y * s.nx + xx;
        double r = b[i];
        // neighbours in ascending index order: -z, -y, -x, +x, +y, +z (a_ij = -T)
        if (s.dim == 3 && z > 0) r = fma(s.Tz[i - sxy], x[i - sxy], r);
        if (y > 0) r = fma(s.Ty[i - s.nx], x[i - s.nx], r);
        if (xx > 0) r = fma(s.Tx[i - 1], x[i - 1], r);
        if (xx + 1 < s.nx) r = fma(s.Tx[i], x[i + 1], r);
        if (y + 1 < s.ny) r = fma(s.Ty[i], x[i + s.nx], r);
        if (s.dim == 3 && z + 1 < s.nz) r = fma(s.Tz[i], x[i + sxy], r);
        x[i] = r / s.D[i];
    }
}

// One colour of a CSR sweep (rows whose colour is c).
__global__ void gs_csr_kernel(Csr cs, const uint8_t *__restrict__ colour, const double *__restrict__ b, double *x,
                              int c) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cs.n; i += (int64_t)gridDim.x * blockDim.x) {
        if (colour[i] != c) continue;
        double r = b[i], d = 0.0;
        const int32_t e1 = cs.rp[i + 1];
        for (int32_t e = cs.rp[i]; e < e1; ++e) {
            const int32_t j = LC_IDX(cs.ci[e], cs.n);
            if (j == i) d = cs.av[e];
            else r = fma(-cs.av[e], x[j], r);
        }
        x[i] = r / d;
    }
}

// Colouring check: colour < ncol, and no stored off-diagonal a_ij != 0 joins
// two rows of the same colour.
__global__ void check_colouring_kernel(Csr cs, const uint8_t *__restrict__ colour, int ncol, int *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cs.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ci_ = colour[i];
        bool ok = ci_ < ncol;
        const int32_t e1 = cs.rp[i + 1];
        for (int32_t e = cs.rp[i]; ok && e < e1; ++e) {
            const int32_t j = cs.ci[e];
            if (j != i && cs.av[e] != 0.0 && colour[j] == ci_) ok = false;
        }
        if (!ok) atomicExch(bad, 1);
    }
}

}  // namespace

cudaError_t launch_gs_stencil(const Stencil &s, const double *b, double *x, int sweeps, cudaStream_t st) {
    const int64_t items = (int64_t)((s.nx + 1) / 2) * s.ny * s.nz;
    const int grid = (int)std::min<int64_t>((items + 255) / 256, 152 * 16);
    for (int sw = 0; sw < sweeps; ++sw)
        for (int c = 0; c < 2; ++c) {
            gs_stencil_kernel<<<grid < 1 ? 1 : grid, 256, 0, st>>>(s, b, x, c);
            note_launches(1);
        }
    return cudaGetLastError();
}

cudaError_t launch_gs_csr(const Csr &cs, const uint8_t *colour, int ncol, const double *b, double *x, int sweeps,
                          cudaStream_t st) {
    const int grid = (int)std::min<int64_t>(((int64_t)cs.n + 255) / 256, 152 * 16);
    for (int sw = 0; sw < sweeps; ++sw)
        for (int c = 0; c < ncol; ++c) {
            gs_csr_kernel<<<grid < 1 ? 1 : grid, 256, 0, st>>>(cs, colour, b, x, c);
            note_launches(1);
        }
    return cudaGetLastError();
}

cudaError_t launch_check_colouring(const Csr &cs, const uint8_t *colour, int ncol, int *bad, cudaStream_t st) {
    const int grid = (int)std::min<int64_t>(((int64_t)cs.n + 255) / 256, 152 * 8);
    check_colouring_kernel<<<grid < 1 ? 1 : grid, 256, 0, st>>>(cs, colour, ncol, bad);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace lc
