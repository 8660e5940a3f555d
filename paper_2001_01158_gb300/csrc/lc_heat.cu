// lc_heat.cu -- the nonlinear 2D heat problem of Sec. 3.2 on the GPU: the
// conductivities kappa = T^p of a Picard iterate, the Picard-linearised
// backward-Euler system (Eq. picard-equs) as a 5-point stencil operator and
// right-hand side, and the norm of a Picard update.  The Picard loop itself
// (lc_heat2d_step in lc_api.cu) calls these and the Alg 1 / PCG solves.
//
// Assembly, per cell P with c = 1/(h h) and faces visited W, E, S, N:
//   interior face   T_f = ((2 kappa_P) kappa_N / (kappa_P + kappa_N)) c
//   Dirichlet side  g   = (2 kappa_P) c     (ghost at half a cell; value to b)
//   Neumann side    no flux
//   D_P = 1/dt, then D_P = D_P + T_f or + g per face
//   b_P = Tn_P (1/dt), then b_P = b_P + g T_side per Dirichlet face
//   Tx_P = T_f of the east face (0 on the last column), Ty_P of the north face.
// Each face is computed by both of its cells with the same rounding
// ((2a) b and (2b) a round the same product), so the operator is exactly
// symmetric.
#include "lc_internal.cuh"

namespace lc {

namespace {

__global__ void heat_kappa_kernel(int64_t n, const double *__restrict__ T, double p, double *kappa) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        kappa[i] = pow(T[i], p);
}

__global__ void heat_assemble_kernel(int nx, int ny, double c, double inv_dt, HeatBc bc,
                                     const double *__restrict__ kappa, const double *__restrict__ Tn, double *D,
                                     double *Tx, double *Ty, double *b) {
    const int64_t n = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        const double kp = kappa[i];
        const int64_t nb[4] = {x > 0 ? i - 1 : -1, x + 1 < nx ? i + 1 : -1, y > 0 ? i - nx : -1,
                               y + 1 < ny ? i + nx : -1};
        // separate roundings (no contraction into FMAs), as the definition reads
        double tf[4];
        double d = inv_dt, bi = __dmul_rn(Tn[i], inv_dt);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            tf[f] = 0.0;
            if (nb[f] >= 0) {
                const double kn = kappa[nb[f]];
                tf[f] = __dmul_rn(__ddiv_rn(__dmul_rn(2.0 * kp, kn), __dadd_rn(kp, kn)), c);
                d = __dadd_rn(d, tf[f]);
            } else if (bc.type[f] == LC_BC_DIRICHLET) {
                const double g = __dmul_rn(2.0 * kp, c);
                d = __dadd_rn(d, g);
                bi = __dadd_rn(bi, __dmul_rn(g, bc.val[f]));
            }
        }
        D[i] = d;
        Tx[i] = tf[1];
        Ty[i] = tf[3];
        b[i] = bi;
    }
}

// sum (x - y)^2: per-block partials, then one block adds them in order
__global__ void diff2_partial_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                                     double *part) {
    __shared__ double red[128];
    double acc[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = x[i] - y[i];
        acc[0] = fma(d, d, acc[0]);
    }
    block_sum<1, double>(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

__global__ void diff2_final_kernel(int nparts, const double *part, double *out) {
    __shared__ double red[128];
    double acc[1] = {0.0};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) acc[0] += part[b];
    block_sum<1, double>(acc, red);
    if (threadIdx.x == 0) *out = acc[0];
}

}  // namespace

cudaError_t launch_heat_kappa(int64_t n, const double *T, double p, double *kappa, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    heat_kappa_kernel<<<grid < 1 ? 1 : grid, 256, 0, s>>>(n, T, p, kappa);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_heat_assemble(int nx, int ny, double h, double dt, const HeatBc &bc, const double *kappa,
                                 const double *Tn, double *D, double *Tx, double *Ty, double *b, cudaStream_t s) {
    const int64_t n = (int64_t)nx * ny;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    const double c = 1.0 / (h * h), inv_dt = 1.0 / dt;
    heat_assemble_kernel<<<grid < 1 ? 1 : grid, 256, 0, s>>>(nx, ny, c, inv_dt, bc, kappa, Tn, D, Tx, Ty, b);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_diff2(int64_t n, const double *x, const double *y, double *part, double *out, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 4);
    diff2_partial_kernel<<<grid < 1 ? 1 : grid, 256, 0, s>>>(n, x, y, part);
    diff2_final_kernel<<<1, 256, 0, s>>>(grid < 1 ? 1 : grid, part, out);
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace lc
