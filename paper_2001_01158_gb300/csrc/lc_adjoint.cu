// lc_adjoint.cu -- operator assembly from per-cell conductivity and the
// adjoint gradient with respect to it (2D, 5-point, finite volumes).
//
// Operator (grid units, backward Euler with step dt):
//   A = I/dt + sum_faces T_f (e_P - e_N)(e_P - e_N)^T + sum_{boundary faces} 2 k_P e_P e_P^T,
//   T_f = 2 k_P k_N / (k_P + k_N)  (harmonic face conductance, Dirichlet ghost
//   half a cell outside every boundary face).
// For a loss L(x) with A x = b and the adjoint A^T lambda = dL/dx (A is
// symmetric), dL/db = lambda and dL/dk = -lambda^T (dA/dk) x, i.e. per cell c
//   dL/dk_c = - sum_{faces (c,N)} 2 k_N^2/(k_c+k_N)^2 (lam_c - lam_N)(x_c - x_N)
//             - sum_{boundary faces of c} 2 lam_c x_c.
#include "lc_internal.cuh"

namespace lc {

namespace {

// D, Tx, Ty of cell i in the order of the seeded generators: face
// conductances (2 kP) kE / (kP + kE); D = 1/dt, then east, west, north,
// south faces, then the ghost terms of the west, east, south, north
// boundaries.
__global__ void assemble_2d_kernel(int nx, int ny, const double *__restrict__ k, double inv_dt,
                                   double *__restrict__ D, double *__restrict__ Tx, double *__restrict__ Ty) {
    const int64_t n = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        const double kp = k[i];
        auto face = [](double a, double b) { return __ddiv_rn(__dmul_rn(__dmul_rn(2.0, a), b), __dadd_rn(a, b)); };
        const double te = x + 1 < nx ? face(kp, k[i + 1]) : 0.0;
        const double tw = x > 0 ? face(k[i - 1], kp) : 0.0;
        const double tn = y + 1 < ny ? face(kp, k[i + nx]) : 0.0;
        const double ts = y > 0 ? face(k[i - nx], kp) : 0.0;
        double d = inv_dt;
        if (x + 1 < nx) d = __dadd_rn(d, te);
        if (x > 0) d = __dadd_rn(d, tw);
        if (y + 1 < ny) d = __dadd_rn(d, tn);
        if (y > 0) d = __dadd_rn(d, ts);
        const double g = __dmul_rn(2.0, kp);
        if (x == 0) d = __dadd_rn(d, g);
        if (x == nx - 1) d = __dadd_rn(d, g);
        if (y == 0) d = __dadd_rn(d, g);
        if (y == ny - 1) d = __dadd_rn(d, g);
        D[i] = d;
        Tx[i] = te;
        Ty[i] = tn;
    }
}

__global__ void adjoint_grad_k_2d_kernel(int nx, int ny, const double *__restrict__ k, const double *__restrict__ x,
                                         const double *__restrict__ lam, double *__restrict__ dk) {
    const int64_t n = (int64_t)nx * ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(c % nx), yy = (int)(c / nx);
        const double kc = k[c], xc = x[c], lc = lam[c];
        double s = 0.0;
        auto nb = [&](bool ok, int64_t m) {
            if (ok) {
                const double km = k[m];
                const double den = kc + km;
                const double dT = 2.0 * km * km / (den * den);
                s = fma(dT * (lc - lam[m]), xc - x[m], s);
            } else {
                s = fma(2.0 * lc, xc, s);
            }
        };
        nb(xx > 0, c - 1);
        nb(xx + 1 < nx, c + 1);
        nb(yy > 0, c - nx);
        nb(yy + 1 < ny, c + nx);
        dk[c] = -s;
    }
}

inline unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_assemble_2d(int nx, int ny, const double *k, double dt, double *D, double *Tx, double *Ty,
                               cudaStream_t s) {
    assemble_2d_kernel<<<grid_for((int64_t)nx * ny), 256, 0, s>>>(nx, ny, k, 1.0 / dt, D, Tx, Ty);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_grad_k_2d(int nx, int ny, const double *k, const double *x, const double *lam, double *dk,
                                     cudaStream_t s) {
    adjoint_grad_k_2d_kernel<<<grid_for((int64_t)nx * ny), 256, 0, s>>>(nx, ny, k, x, lam, dk);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace lc
