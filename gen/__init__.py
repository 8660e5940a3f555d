"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module only builds problem data: conductivity fields, the backward-Euler
diffusion operator assembled from them (in stencil and CSR form), sources,
right-hand sides and initial iterates.  It contains none of the local
character-based method itself (no residual marking, no expansion, no
extraction, no Krylov solve), so both sides of every parity test can take
their inputs from here without sharing any of the method's arithmetic.

Operator (finite volumes, grid units h = 1, backward Euler with step dt):

    A = I/dt + sum_faces T_f (e_P - e_N)(e_P - e_N)^T + sum_{boundary faces} 2 k_P e_P e_P^T

with the harmonic face conductance T_f = 2 k_P k_N / (k_P + k_N) and a
homogeneous Dirichlet ghost half a cell outside every boundary face.  A is
symmetric and strictly diagonally dominant with a positive diagonal, hence
SPD, for any dt > 0.

Stencil layout (structure-of-arrays, row-major cell index
i = x + nx*(y + ny*z)):
    D[i]   diagonal a_ii
    Tx[i]  conductance of the face between i and i+1       (a_{i,i+1} = -Tx[i])
    Ty[i]  conductance of the face between i and i+nx      (a_{i,i+nx} = -Ty[i])
    Tz[i]  conductance of the face between i and i+nx*ny   (a_{i,i+nx*ny} = -Tz[i])
Entries of Tx/Ty/Tz on the last column/row/plane (no face) are 0 and unused.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Stencil", "operator_2d", "operator_3d", "stencil_to_csr", "csr_matvec",
    "cfg1_heat2d", "cfg2_fronts2d", "cfg3_aniso3d", "cfg4_batch", "cfg5_adjoint",
    "random_stencil_2d", "random_stencil_3d", "example1",
]


@dataclass
class Stencil:
    """A 2D (nz == 1, Tz None) or 3D structured operator in SoA form."""
    shape: tuple            # (nx, ny, nz)
    D: np.ndarray
    Tx: np.ndarray
    Ty: np.ndarray
    Tz: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return 2 if self.Tz is None else 3

    @property
    def n(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz


def _harmonic(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return (2.0 * a) * b / (a + b)


def operator_2d(k: np.ndarray, dt: float = 1.0) -> Stencil:
    """Assemble the 5-point operator for a cell conductivity field k[ny, nx]."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    ny, nx = k.shape
    Tx = np.zeros_like(k)
    Ty = np.zeros_like(k)
    if nx > 1:
        Tx[:, :-1] = _harmonic(k[:, :-1], k[:, 1:])
    if ny > 1:
        Ty[:-1, :] = _harmonic(k[:-1, :], k[1:, :])
    D = np.full_like(k, 1.0 / dt)
    D[:, :-1] += Tx[:, :-1]
    D[:, 1:] += Tx[:, :-1]
    D[:-1, :] += Ty[:-1, :]
    D[1:, :] += Ty[:-1, :]
    D[:, 0] += 2.0 * k[:, 0]
    D[:, -1] += 2.0 * k[:, -1]
    D[0, :] += 2.0 * k[0, :]
    D[-1, :] += 2.0 * k[-1, :]
    return Stencil((nx, ny, 1), D.ravel(), Tx.ravel(), Ty.ravel(), None, {"dt": dt})


def operator_3d(kx: np.ndarray, ky: np.ndarray, kz: np.ndarray, dt: float = 1.0) -> Stencil:
    """Assemble the 7-point operator for per-direction conductivities k_d[nz, ny, nx]."""
    kx, ky, kz = (np.ascontiguousarray(a, dtype=np.float64) for a in (kx, ky, kz))
    nz, ny, nx = kx.shape
    Tx = np.zeros_like(kx)
    Ty = np.zeros_like(kx)
    Tz = np.zeros_like(kx)
    if nx > 1:
        Tx[:, :, :-1] = _harmonic(kx[:, :, :-1], kx[:, :, 1:])
    if ny > 1:
        Ty[:, :-1, :] = _harmonic(ky[:, :-1, :], ky[:, 1:, :])
    if nz > 1:
        Tz[:-1, :, :] = _harmonic(kz[:-1, :, :], kz[1:, :, :])
    D = np.full_like(kx, 1.0 / dt)
    D[:, :, :-1] += Tx[:, :, :-1]
    D[:, :, 1:] += Tx[:, :, :-1]
    D[:, :-1, :] += Ty[:, :-1, :]
    D[:, 1:, :] += Ty[:, :-1, :]
    D[:-1, :, :] += Tz[:-1, :, :]
    D[1:, :, :] += Tz[:-1, :, :]
    D[:, :, 0] += 2.0 * kx[:, :, 0]
    D[:, :, -1] += 2.0 * kx[:, :, -1]
    D[:, 0, :] += 2.0 * ky[:, 0, :]
    D[:, -1, :] += 2.0 * ky[:, -1, :]
    D[0, :, :] += 2.0 * kz[0, :, :]
    D[-1, :, :] += 2.0 * kz[-1, :, :]
    return Stencil((nx, ny, nz), D.ravel(), Tx.ravel(), Ty.ravel(), Tz.ravel(), {"dt": dt})


def stencil_to_csr(op: Stencil):
    """CSR (int32 rowptr, int32 col ascending per row, float64 val) of a stencil.

    Off-diagonals are the negated face conductances (negation is exact), one
    entry per interior face; rows list their entries in ascending column order
    (-z, -y, -x, P, +x, +y, +z).
    """
    nx, ny, nz = op.shape
    n = op.n
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    cand_col, cand_val, cand_ok = [], [], []

    def add(ok, col, val):
        cand_ok.append(ok)
        cand_col.append(np.where(ok, col, 0))
        cand_val.append(np.where(ok, val, 0.0))

    sxy = nx * ny
    if op.dim == 3:
        add(z > 0, idx - sxy, -op.Tz[np.maximum(idx - sxy, 0)])
    add(y > 0, idx - nx, -op.Ty[np.maximum(idx - nx, 0)])
    add(x > 0, idx - 1, -op.Tx[np.maximum(idx - 1, 0)])
    add(np.ones(n, bool), idx, op.D)
    add(x < nx - 1, idx + 1, -op.Tx)
    add(y < ny - 1, idx + nx, -op.Ty)
    if op.dim == 3:
        add(z < nz - 1, idx + sxy, -op.Tz)
    ok = np.stack(cand_ok, 1)
    col = np.stack(cand_col, 1)[ok].astype(np.int32)
    val = np.stack(cand_val, 1)[ok].astype(np.float64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(ok.sum(1), out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    return rowptr.astype(np.int32), col, val


def stencil_matvec(op: "Stencil", x: np.ndarray) -> np.ndarray:
    """y = A x for a stencil operator, vectorised over the grid (problem set-up)."""
    nx, ny, nz = op.shape
    X = np.asarray(x, dtype=np.float64).reshape(nz, ny, nx)
    D = op.D.reshape(nz, ny, nx)
    Tx = op.Tx.reshape(nz, ny, nx)
    Ty = op.Ty.reshape(nz, ny, nx)
    y = D * X
    y[:, :, :-1] -= Tx[:, :, :-1] * X[:, :, 1:]
    y[:, :, 1:] -= Tx[:, :, :-1] * X[:, :, :-1]
    y[:, :-1, :] -= Ty[:, :-1, :] * X[:, 1:, :]
    y[:, 1:, :] -= Ty[:, :-1, :] * X[:, :-1, :]
    if op.Tz is not None:
        Tz = op.Tz.reshape(nz, ny, nx)
        y[:-1] -= Tz[:-1] * X[1:]
        y[1:] -= Tz[:-1] * X[:-1]
    return y.ravel()


def redblack_colouring(shape) -> np.ndarray:
    """Colour (x + y + z) mod 2 of every cell, i = x + nx (y + ny z): no two
    cells of the 5-point / 7-point stencil that are neighbours share a colour."""
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((x + y + z) & 1).astype(np.uint8).ravel()


def csr_matvec(rowptr, col, val, x):
    """y = A x for problem set-up (manufactured right-hand sides)."""
    import scipy.sparse as sp
    n = len(rowptr) - 1
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    return A @ x


def _centres(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def _disc(nx: int, ny: int, cx: float, cy: float, radius: float) -> np.ndarray:
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    return (((xx - cx) ** 2 + (yy - cy) ** 2) <= radius * radius).astype(np.float64)


def _k_sine(n: int) -> np.ndarray:
    c = _centres(n)
    return 1.0 + 0.5 * np.outer(np.sin(2 * math.pi * c), np.sin(2 * math.pi * c))


def _smooth_field(n_x: int, n_y: int, rng) -> np.ndarray:
    cx, cy = _centres(n_x), _centres(n_y)
    f = np.ones((n_y, n_x))
    for _ in range(4):
        p, q = rng.integers(1, 4, size=2)
        a = rng.uniform(-0.25, 0.25)
        f += a * np.outer(np.sin(math.pi * q * cy), np.sin(math.pi * p * cx))
    return f


def cfg1_heat2d(seed: int = 0, n: int = 128, radius: float = 10.0, dt: float = 1.0, literal: bool = False):
    """2D heat step: k = 1 + 0.5 sin(2 pi x) sin(2 pi y); smooth seeded previous
    solution x_prev; new unit source in a seeded disc.  The time-stepped
    reading sets b = A x_prev + s (x_prev solved the previous step), so that
    r0 = b - A x_prev equals the source up to rounding; literal=True gives
    b = x_prev/dt + s instead."""
    rng = np.random.default_rng(seed)
    op = operator_2d(_k_sine(n), dt)
    x_prev = _smooth_field(n, n, rng).ravel()
    lo, hi = int(round(20 * n / 128)), int(round(107 * n / 128))
    c = rng.integers(lo, max(hi, lo) + 1, size=2)
    s = _disc(n, n, float(c[0]), float(c[1]), radius).ravel()
    if literal:
        b = x_prev / dt + s
    else:
        b = stencil_matvec(op, x_prev) + s
    return {"op": op, "b": b, "x0": x_prev, "source": s, "centre": c}


@dataclass
class FrontSequence:
    """2D moving Gaussian front: b^n = x^{n-1}/dt + s^n."""
    op: Stencil
    n: int
    steps: int
    c0: np.ndarray
    theta: float
    width: float
    speed: float

    def source(self, step: int) -> np.ndarray:
        c = self.c0 + self.speed * step * np.array([math.cos(self.theta), math.sin(self.theta)])
        yy = np.arange(self.n, dtype=np.float64)[:, None]
        xx = np.arange(self.n, dtype=np.float64)[None, :]
        d2 = (xx - c[0]) ** 2 + (yy - c[1]) ** 2
        return np.exp(-d2 / (2.0 * self.width * self.width)).ravel()


def cfg2_fronts2d(seed: int = 0, n: int = 2048, steps: int = 20, n_rect: int = 64,
                  side=(16, 256), width: float = 30.0, speed: float = 8.0, dt: float = 1.0):
    """2D diffusion with discontinuous conductivity: background 1 plus n_rect
    seeded rectangles (side ~ U{16..256}, later ones overwrite) with
    k = 10^U(0,3); a Gaussian front (sigma = width cells) moving speed cells
    per step.  x^0 = 0; step n solves A x^n = x^{n-1}/dt + s^n."""
    rng = np.random.default_rng(seed)
    k = np.ones((n, n))
    scale = n / 2048.0
    for _ in range(n_rect):
        w, h = (max(1, int(round(v * scale))) for v in rng.integers(side[0], side[1] + 1, size=2))
        x0 = int(rng.integers(0, max(1, n - w + 1)))
        y0 = int(rng.integers(0, max(1, n - h + 1)))
        k[y0:y0 + h, x0:x0 + w] = 10.0 ** rng.uniform(0.0, 3.0)
    op = operator_2d(k, dt)
    c0 = rng.uniform(400 * scale, 1648 * scale, size=2)
    theta = float(rng.uniform(0.0, 2 * math.pi))
    seq = FrontSequence(op, n, steps, c0, theta, width * scale if n < 2048 else width, speed * scale if n < 2048 else speed)
    return {"op": op, "seq": seq, "k": k}


def cfg3_aniso3d(seed: int = 0, n: int = 256, box: int = 20, sigma: float = 0.5, ratios=(1.0, 10.0, 100.0), dt: float = 1.0):
    """3D 7-point anisotropic diffusion: k_d = ratio_d * exp(sigma * z_c), z_c iid
    N(0,1) per cell; unit source on a seeded box; x^0 = 0, b = s."""
    rng = np.random.default_rng(seed)
    m = np.exp(sigma * rng.standard_normal((n, n, n)))
    op = operator_3d(ratios[0] * m, ratios[1] * m, ratios[2] * m, dt)
    bx = min(box, n)
    c = rng.integers(0, n - bx + 1, size=3)
    s = np.zeros((n, n, n))
    s[c[2]:c[2] + bx, c[1]:c[1] + bx, c[0]:c[0] + bx] = 1.0
    s = s.ravel()
    return {"op": op, "b": s.copy(), "x0": np.zeros(n ** 3), "source": s, "corner": c}


def cfg4_batch(seed: int = 0, count: int = 512, nmin: int = 64, nmax: int = 512, eta=(0.01, 0.30)):
    """Many independent 2D systems like cfg1, side log-uniform in [nmin, nmax],
    each with its own seed and a disc source sized so that roughly a fraction
    eta_s ~ U(eta) of the cells changes."""
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))).astype(int)
    etas = rng.uniform(eta[0], eta[1], size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    out = []
    for ns, es, sd in zip(sides, etas, seeds):
        radius = max(1.0, math.sqrt(es * ns * ns / math.pi) - 2.0)
        out.append(cfg1_heat2d(int(sd), int(ns), radius=radius))
    return out


def cfg5_adjoint(seed: int = 0, n: int = 1024, radius: float = 80.0, dt: float = 1.0, modes: int = 8):
    """Adjoint workload: k as cfg1; k_target = k * exp(0.3 G) with G a sum of
    `modes` seeded Fourier modes; b = x_prev/dt + s with a disc source."""
    rng = np.random.default_rng(seed)
    k = _k_sine(n)
    c = _centres(n)
    G = np.zeros((n, n))
    for _ in range(modes):
        p, q = rng.integers(1, 6, size=2)
        a = rng.uniform(-1.0, 1.0)
        ph = rng.uniform(0, 2 * math.pi, size=2)
        G += a * np.outer(np.cos(math.pi * q * c + ph[1]), np.cos(math.pi * p * c + ph[0]))
    G /= max(1.0, float(np.abs(G).max()))
    k_target = k * np.exp(0.3 * G)
    x_prev = _smooth_field(n, n, rng).ravel()
    cc = rng.uniform(0.3 * n, 0.7 * n, size=2)
    s = _disc(n, n, cc[0], cc[1], radius * n / 1024.0).ravel()
    b = x_prev / dt + s
    return {"k": k, "k_target": k_target, "b": b, "dt": dt, "n": n}


def mg_standin(seed: int = 0, groups: int = 64, nx: int = 88, ny: int = 80, dt: float = 1.0,
               hot_radius: float = 6.0, shift: float = 2.0):
    """Multi-group radiation-diffusion stand-in (the structure of Sec. 3.3's
    systems on synthetic data): `groups` 5-point systems on one nx x ny mesh
    (88 x 80 = 7040 cells, the paper's cell count) with the same sparsity
    pattern and group-dependent coefficients.  A smooth density rho and an
    electron temperature Te with a hot spot give Kramers-like cross sections
    sigma_g = rho nu_g^-3 / sqrt(Te) over log-spaced group energies nu_g;
    diffusion coefficients kappa_g = 1/(3 sigma_g); A_g = operator_2d(kappa_g,
    dt) plus sigma_g on the diagonal (absorption).  Between two source
    iterations the hot spot moves by `shift` cells, so the emission
    4 pi sigma_g B_g changes only near it: x0_g is the previous iterate (a
    smooth field), b_g = A_g x0_g + 4 pi sigma_g (B_g(Te_new) - B_g(Te_old)).
    B_g(T) = T^4 nu_g^3 / (exp(nu_g / T) - 1) (Planck shape, arbitrary units)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * xx / nx + rng.uniform(0, 6.3)) * np.cos(2 * np.pi * yy / ny)
    c = np.array([rng.uniform(0.3, 0.7) * nx, rng.uniform(0.3, 0.7) * ny])
    ang = rng.uniform(0, 2 * np.pi)
    c_new = c + shift * np.array([math.cos(ang), math.sin(ang)])

    def temperature(cc):
        return 0.1 + 0.9 * np.exp(-((xx - cc[0]) ** 2 + (yy - cc[1]) ** 2) / (2.0 * hot_radius ** 2))

    te_old, te_new = temperature(c), temperature(c_new)
    nu = np.logspace(-1.0, 1.0, groups)
    out = []
    for g in range(groups):
        sigma = rho * nu[g] ** -3 / np.sqrt(te_old)
        op = operator_2d(1.0 / (3.0 * sigma), dt)
        op.D += sigma.ravel()

        def planck(t):
            return t ** 4 * nu[g] ** 3 / np.expm1(nu[g] / t)

        x0 = (planck(te_old) / planck(te_old).max()).ravel()
        emis = 4.0 * np.pi * sigma * (planck(te_new) - planck(te_old))
        out.append({"op": op, "x0": x0, "b": stencil_matvec(op, x0) + emis.ravel(), "nu": float(nu[g])})
    return out


def _csr_from_coo(n, rows, cols, vals):
    """Sorted, duplicate-summed CSR (int32 indices, FP64 values) of COO triplets."""
    import scipy.sparse as sp
    M = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return (M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


def _ninepoint_edges(rng, nx: int, ny: int, k: np.ndarray, shear: np.ndarray):
    """Edges (i, j, w) of a 9-point stencil on an nx x ny grid: axis faces with
    the harmonic mean of k, diagonals with a fraction |shear| of it (the
    cross terms a distorted quadrilateral mesh produces); all w > 0."""
    idx = np.arange(nx * ny).reshape(ny, nx)
    out_i, out_j, out_w = [], [], []

    def add(a, b, w):
        out_i.append(a.ravel()); out_j.append(b.ravel()); out_w.append(w.ravel())

    kk = k.reshape(ny, nx)
    sh = shear.reshape(ny, nx)
    add(idx[:, :-1], idx[:, 1:], _harmonic(kk[:, :-1], kk[:, 1:]) * (1.0 - 0.5 * np.abs(sh[:, :-1])))
    add(idx[:-1, :], idx[1:, :], _harmonic(kk[:-1, :], kk[1:, :]) * (1.0 - 0.5 * np.abs(sh[:-1, :])))
    add(idx[:-1, :-1], idx[1:, 1:], 0.5 * _harmonic(kk[:-1, :-1], kk[1:, 1:]) * np.maximum(sh[:-1, :-1], 0.0) + 1e-3)
    add(idx[:-1, 1:], idx[1:, :-1], 0.5 * _harmonic(kk[:-1, 1:], kk[1:, :-1]) * np.maximum(-sh[:-1, 1:], 0.0) + 1e-3)
    return np.concatenate(out_i), np.concatenate(out_j), np.concatenate(out_w)


def _laplacian_coo(n, ei, ej, ew, diag):
    rows = np.concatenate([ei, ej, ei, ej, np.arange(n)])
    cols = np.concatenate([ej, ei, ei, ej, np.arange(n)])
    vals = np.concatenate([-ew, -ew, ew, ew, diag])
    return rows, cols, vals


def ninepoint_2d(seed: int, nx: int, ny: int, dt: float = 1.0, kmax: float = 100.0):
    """A 9-point diffusion operator as a general CSR matrix (the pattern of the
    paper's deforming-mesh systems, Sec. 3.3): k log-uniform in [1, kmax],
    a smooth random mesh shear in [-0.8, 0.8] weighting the diagonal
    couplings; A = I/dt + sum_e w_e (e_i - e_j)(e_i - e_j)^T + a Dirichlet
    ghost 2 k on the outer faces.  Symmetric, strictly diagonally dominant,
    SPD.  Returns (rowptr, col, val)."""
    rng = np.random.default_rng(seed)
    n = nx * ny
    k = 10.0 ** rng.uniform(0.0, math.log10(kmax), n)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 2)
    shear = (0.8 * np.sin(2 * np.pi * xx / max(nx, 2) + ph[0]) * np.cos(2 * np.pi * yy / max(ny, 2) + ph[1])).ravel()
    ei, ej, ew = _ninepoint_edges(rng, nx, ny, k, shear)
    diag = np.full(n, 1.0 / dt)
    kk = k.reshape(ny, nx)
    ghost = np.zeros((ny, nx))
    ghost[:, 0] += 2 * kk[:, 0]; ghost[:, -1] += 2 * kk[:, -1]; ghost[0, :] += 2 * kk[0, :]; ghost[-1, :] += 2 * kk[-1, :]
    return _csr_from_coo(n, *_laplacian_coo(n, ei, ej, ew, diag + ghost.ravel()))


def threeT_2d(seed: int, nx: int, ny: int, dt: float = 1.0):
    """A 3T-like coupled system (radiation, electron and ion temperatures per
    cell, interleaved: unknown 3 c + v), the coupled 3 x 3 block rows of the
    paper's 3T systems (Sec. 3.4) on synthetic data: three 9-point diffusion
    operators with conductivities of very different size (radiation 1..1e3,
    electron 1..10, ion 1e-3..1e-2) plus per-cell energy exchange
    w_er (T_e - T_r)^2 + w_ei (T_e - T_i)^2 terms (w log-uniform): symmetric,
    SPD.  Returns (rowptr, col, val)."""
    rng = np.random.default_rng(seed)
    nc = nx * ny
    n = 3 * nc
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 2)
    shear = (0.6 * np.sin(2 * np.pi * xx / max(nx, 2) + ph[0]) * np.cos(2 * np.pi * yy / max(ny, 2) + ph[1])).ravel()
    rows, cols, vals = [], [], []
    for v, (lo, hi) in enumerate([(0.0, 3.0), (0.0, 1.0), (-3.0, -2.0)]):
        k = 10.0 ** rng.uniform(lo, hi, nc)
        ei, ej, ew = _ninepoint_edges(rng, nx, ny, k, shear)
        kk = k.reshape(ny, nx)
        ghost = np.zeros((ny, nx))
        ghost[:, 0] += 2 * kk[:, 0]; ghost[:, -1] += 2 * kk[:, -1]; ghost[0, :] += 2 * kk[0, :]; ghost[-1, :] += 2 * kk[-1, :]
        r, c, w = _laplacian_coo(nc, ei, ej, ew, np.full(nc, 1.0 / dt) + ghost.ravel())
        rows.append(3 * r + v); cols.append(3 * c + v); vals.append(w)
    cell = np.arange(nc)
    for (a, b), (lo, hi) in [((1, 0), (0.0, 2.0)), ((1, 2), (-1.0, 1.0))]:
        w = 10.0 ** rng.uniform(lo, hi, nc)
        ei, ej = 3 * cell + a, 3 * cell + b
        rows.append(np.concatenate([ei, ej, ei, ej]))
        cols.append(np.concatenate([ej, ei, ei, ej]))
        vals.append(np.concatenate([-w, -w, w, w]))
    return _csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def greedy_colouring(rowptr, col) -> np.ndarray:
    """Smallest colour not taken by an earlier neighbour, rows in ascending
    order: a proper colouring for multicolour Gauss-Seidel on a CSR pattern."""
    n = len(rowptr) - 1
    colour = np.zeros(n, np.uint8)
    for i in range(n):
        taken = set(colour[col[rowptr[i]:rowptr[i + 1]][col[rowptr[i]:rowptr[i + 1]] < i]].tolist())
        c = 0
        while c in taken:
            c += 1
        colour[i] = c
    return colour


def random_stencil_2d(seed: int, nx: int, ny: int, dt: float = 1.0, kmax: float = 100.0) -> Stencil:
    """Small random 5-point operator (k log-uniform in [1, kmax]) for tests."""
    rng = np.random.default_rng(seed)
    k = np.exp(rng.uniform(0.0, math.log(kmax), size=(ny, nx)))
    return operator_2d(k, dt)


def random_stencil_3d(seed: int, nx: int, ny: int, nz: int, dt: float = 1.0, kmax: float = 100.0) -> Stencil:
    """Small random anisotropic 7-point operator for tests."""
    rng = np.random.default_rng(seed)
    kx, ky, kz = (np.exp(rng.uniform(0.0, math.log(kmax), size=(nz, ny, nx))) for _ in range(3))
    return operator_3d(kx, ky, kz, dt)


def example1():
    """The 9x9 tridiagonal system of the paper's Example 1 (Sec. 2.3): unit
    diagonal, off-diagonals a_{i,i+1} = a_{i+1,i} = -1/(i+1) (1-based i),
    x_i = 10^-i, x0 = (1, 0.1, 1.001e-3, ..., 1.001e-9), b = A x."""
    n = 9
    A = np.eye(n)
    for i in range(1, n):
        A[i - 1, i] = A[i, i - 1] = -1.0 / (i + 1)
    x = np.array([10.0 ** -(i + 1) for i in range(n)])
    x0 = np.array([1.0, 1e-1] + [1.001 * 10.0 ** -(i + 1) for i in range(2, n)])
    b = A @ x
    rowptr, col, val = [0], [], []
    for i in range(n):
        for j in range(n):
            if A[i, j] != 0.0:
                col.append(j)
                val.append(A[i, j])
        rowptr.append(len(col))
    return {"A": A, "x": x, "x0": x0, "b": b,
            "rowptr": np.array(rowptr, np.int32), "col": np.array(col, np.int32), "val": np.array(val)}
