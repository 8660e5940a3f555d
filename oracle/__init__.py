"""Oracle: plain serial FP64 CPU reference of the local character-based solve.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it never calls the CUDA library: the two share no code,
only the seeded inputs of :mod:`gen`.

The arithmetic lives in ``lc_oracle.c`` (plain loops, -ffp-contract=off);
this module compiles it with gcc on first use and wraps it with ctypes and
NumPy.  Each function names the passage of Ye, An & Xu (arXiv 2001.01158) it
follows; the readings of points the paper leaves open are listed at the top
of ``lc_oracle.c``.

Pins (tests/test_oracle_*.py) tie each function to something other than
itself: Example 1's printed trace, dense LU, brute-force NumPy set
definitions on tiny inputs, closed forms and invariants.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

THR_EPS_NORMB, THR_REL_MAX = 0, 1
EXP_NONE, EXP_DILATE, EXP_PAPER = 0, 1, 2
MARK_RESIDUAL, MARK_GRADIENT = 0, 1
OK, NOT_CONVERGED, BREAKDOWN = 0, 4, 5

_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


class _Params(C.Structure):
    _fields_ = [("mark_mode", C.c_int32), ("thr_mode", C.c_int32), ("thr_param", C.c_double),
                ("exp_mode", C.c_int32), ("exp_rounds", C.c_int32), ("alpha", C.c_double),
                ("grad_layers", C.c_int32), ("tol", C.c_double), ("tol_local", C.c_double),
                ("maxit", C.c_int32), ("gs_sweeps", C.c_int32), ("gs_ncolours", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("K", C.c_int32), ("nnzB", C.c_int32), ("it_local", C.c_int32),
                ("it_global", C.c_int32), ("early_exit", C.c_int32), ("status", C.c_int32),
                ("tau", C.c_double), ("relres_tilde", C.c_double), ("relres_final", C.c_double)]


class _HeatStats(C.Structure):
    _fields_ = [("picard_its", C.c_int32), ("it_local", C.c_int32), ("it_global", C.c_int32),
                ("K_sum", C.c_int32), ("early_exits", C.c_int32), ("status", C.c_int32),
                ("last_update", C.c_double)]


BC_DIRICHLET, BC_NEUMANN = 0, 1


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        _lib = load(build_oracle())
    return _lib


def threads() -> int:
    """Threads the loaded oracle library's loops use (1: the serial oracle)."""
    return int(lib().orc_threads())


@contextlib.contextmanager
def openmp_build():
    """Within this block every function of this module runs on the
    timing-only OpenMP build of the oracle source (row loops in parallel on
    all host cores, dot products as OpenMP reductions: another rounding
    order).  For CPU-baseline timing only; parity uses the serial build."""
    global _lib
    saved = lib()
    _lib = load(build_oracle(openmp=True))
    try:
        yield _lib
    finally:
        _lib = saved


def load(path: str):
    """Open an oracle shared library at `path` and declare its signatures."""
    L = C.CDLL(path)
    csr = [C.c_int32, _i32p, _i32p, _f64p]
    L.orc_residual.argtypes = csr + [_f64p, _f64p, _f64p]
    L.orc_sumsq.argtypes = [C.c_int32, _f64p]
    L.orc_sumsq.restype = C.c_double
    L.orc_tau_eps_normb.argtypes = [C.c_int32, _f64p, C.c_double]
    L.orc_tau_eps_normb.restype = C.c_double
    L.orc_dilate.argtypes = csr + [_u8p, C.c_int32]
    L.orc_expand_paper.argtypes = csr + [_f64p, _f64p, C.c_double, _u8p, C.c_int32, _f64p]
    L.orc_expand_paper.restype = C.c_int32
    L.orc_mark_residual.argtypes = csr + [_f64p, _f64p, C.c_int32, C.c_double, C.c_int32, C.c_int32,
                                          _u8p, _f64p, C.POINTER(C.c_double), C.POINTER(C.c_int32)]
    L.orc_mark_residual.restype = C.c_int32
    L.orc_gradient.argtypes = csr + [_f64p, _f64p]
    L.orc_mark_gradient.argtypes = csr + [_f64p, C.c_double, C.c_int32, _u8p, _f64p, C.POINTER(C.c_double)]
    L.orc_mark_gradient.restype = C.c_int32
    L.orc_extract.argtypes = csr + [_u8p, _f64p, _f64p, _i32p, _i32p, _i32p, _i32p, _f64p, _f64p, _f64p,
                                    C.POINTER(C.c_int32)]
    L.orc_extract.restype = C.c_int32
    L.orc_assemble.argtypes = [C.c_int32, _f64p, C.c_int32, _i32p, _f64p, _f64p]
    L.orc_threads.argtypes = []
    L.orc_threads.restype = C.c_int32
    L.orc_relres.argtypes = csr + [_f64p, _f64p]
    L.orc_relres.restype = C.c_double
    L.orc_pcg.argtypes = csr + [_f64p, _f64p, C.c_double, C.c_int32, C.POINTER(C.c_int32),
                                C.POINTER(C.c_double)]
    L.orc_pcg.restype = C.c_int32
    L.orc_solve_local_then_global.argtypes = csr + [_f64p, _f64p, C.POINTER(_Params), C.POINTER(_Stats), _u8p,
                                                    _u8p]
    L.orc_solve_local_then_global.restype = C.c_int32
    L.orc_gs_sweep.argtypes = csr + [_f64p, _f64p, _u8p, C.c_int32]
    L.orc_heat2d_system.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, _i32p, _f64p, _f64p, _f64p,
                                    _i32p, _i32p, _f64p, _f64p]
    L.orc_heat2d_system.restype = C.c_int32
    L.orc_heat2d_step.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, _i32p, _f64p, _f64p,
                                  _f64p, C.c_int32, C.POINTER(_Params), C.c_double, C.c_int32,
                                  C.POINTER(_HeatStats), _u8p]
    L.orc_heat2d_step.restype = C.c_int32
    L.orc_adjoint_grad_k_2d.argtypes = [C.c_int32, C.c_int32, _f64p, _f64p, _f64p, _f64p]
    return L


@dataclass
class CSR:
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def n(self) -> int:
        return len(self.rowptr) - 1

    def args(self):
        return (C.c_int32(self.n), self.rowptr, self.col, self.val)

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            for e in range(self.rowptr[i], self.rowptr[i + 1]):
                A[i, self.col[e]] = self.val[e]
        return A


def csr(rowptr, col, val) -> CSR:
    return CSR(np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(col, np.int32),
               np.ascontiguousarray(val, np.float64))


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def residual(A: CSR, b, x) -> np.ndarray:
    """r = b - A x in the canonical order (Alg 3, step 4)."""
    r = np.empty(A.n)
    lib().orc_residual(*A.args(), _f(b), _f(x), r)
    return r


def sumsq(b) -> float:
    """sum b_i^2 in the canonical tree order (threshold of Sec. 2.3.1)."""
    b = _f(b)
    return lib().orc_sumsq(len(b), b)


def tau_eps_normb(b, eps: float) -> float:
    """tau = eps ||b||_2 / sqrt(N) (Sec. 2.3.1)."""
    b = _f(b)
    return lib().orc_tau_eps_normb(len(b), b, eps)


def dilate(A: CSR, mask, layers: int) -> np.ndarray:
    m = np.ascontiguousarray(mask, np.uint8).copy()
    lib().orc_dilate(*A.args(), m, layers)
    return m


def expand_paper(A: CSR, r0, x0, tau: float, mask, emax: int):
    """Alg 3's expansion rounds.  Returns (mask, rounds that added points,
    c) with c[m, j] the quantity tested for candidate j in round m (NaN for
    non-candidates)."""
    m = np.ascontiguousarray(mask, np.uint8).copy()
    c = np.empty(max(emax, 1) * A.n)
    rounds = lib().orc_expand_paper(*A.args(), _f(r0), _f(x0), tau, m, emax, c)
    return m, rounds, c[:emax * A.n].reshape(emax, A.n)


def mark_residual(A: CSR, b, x0, thr_mode=THR_REL_MAX, param=1e-3, exp_mode=EXP_DILATE, rounds=2):
    """Residual-based local domain (Alg 3 and its relative-threshold /
    dilation variant).  Returns dict(mask, r, tau, K, rounds)."""
    mask = np.zeros(A.n, np.uint8)
    r = np.empty(A.n)
    tau = C.c_double()
    done = C.c_int32()
    K = lib().orc_mark_residual(*A.args(), _f(b), _f(x0), thr_mode, param, exp_mode, rounds,
                                mask, r, C.byref(tau), C.byref(done))
    return {"mask": mask, "r": r, "tau": tau.value, "K": K, "rounds": done.value}


def gradient(A: CSR, x) -> np.ndarray:
    """g_i of Eq. grad."""
    g = np.empty(A.n)
    lib().orc_gradient(*A.args(), _f(x), g)
    return g


def mark_gradient(A: CSR, x0, alpha: float, layers: int = 0):
    """Alg 2 (+ optional dilation).  Returns dict(mask, g, gmax, K)."""
    mask = np.zeros(A.n, np.uint8)
    g = np.empty(A.n)
    gmax = C.c_double()
    K = lib().orc_mark_gradient(*A.args(), _f(x0), alpha, layers, mask, g, C.byref(gmax))
    return {"mask": mask, "g": g, "gmax": gmax.value, "K": K}


def extract(A: CSR, mask, b, x0):
    """Local subsystem of Eq. loc-equ.  Returns dict(K, g2l, l2g, B (CSR), rhs, xL0)."""
    n = A.n
    nnz = int(A.rowptr[-1])
    g2l = np.empty(n, np.int32)
    l2g = np.zeros(max(n, 1), np.int32)
    brp = np.zeros(n + 1, np.int32)
    bci = np.zeros(max(nnz, 1), np.int32)
    bav = np.zeros(max(nnz, 1))
    rhs = np.zeros(max(n, 1))
    xl = np.zeros(max(n, 1))
    nzb = C.c_int32()
    K = lib().orc_extract(*A.args(), np.ascontiguousarray(mask, np.uint8), _f(b), _f(x0),
                          g2l, l2g, brp, bci, bav, rhs, xl, C.byref(nzb))
    nz = nzb.value
    return {"K": K, "g2l": g2l, "l2g": l2g[:K].copy(),
            "B": csr(brp[:K + 1].copy(), bci[:nz].copy(), bav[:nz].copy()),
            "rhs": rhs[:K].copy(), "xL0": xl[:K].copy()}


def assemble(x0, l2g, xbar) -> np.ndarray:
    """Eq. sol-assemble."""
    x0 = _f(x0)
    out = np.empty_like(x0)
    l2g = np.ascontiguousarray(l2g, np.int32)
    lib().orc_assemble(len(x0), x0, len(l2g), l2g if len(l2g) else np.zeros(1, np.int32), _f(xbar) if len(l2g) else np.zeros(1), out)
    return out


def relres(A: CSR, b, x) -> float:
    """||b - A x||_2 / ||b||_2."""
    return lib().orc_relres(*A.args(), _f(b), _f(x))


def pcg(A: CSR, b, x0, tol=1e-8, maxit=100000):
    """Jacobi-PCG from x0.  Returns (x, status, iterations, relres)."""
    x = _f(x0).copy()
    it = C.c_int32()
    rr = C.c_double()
    st = lib().orc_pcg(*A.args(), _f(b), x, tol, maxit, C.byref(it), C.byref(rr))
    return x, st, it.value, rr.value


def gs_sweep(A: CSR, b, x, colour, ncolours: int | None = None) -> np.ndarray:
    """One multicolour Gauss-Seidel sweep (Alg 1 step 7) from x; returns the new x."""
    colour = np.ascontiguousarray(colour, dtype=np.uint8)
    nc = int(colour.max()) + 1 if ncolours is None and len(colour) else (ncolours or 0)
    out = _f(x).copy()
    lib().orc_gs_sweep(*A.args(), _f(b), out, colour if len(colour) else np.zeros(1, np.uint8), nc)
    return out


def solve_local_then_global(A: CSR, b, x0, mark_mode=MARK_RESIDUAL, thr_mode=THR_REL_MAX, thr_param=1e-3,
                            exp_mode=EXP_DILATE, exp_rounds=2, alpha=1e-3, grad_layers=0,
                            tol=1e-8, tol_local=None, maxit=100000, gs_sweeps=0, colour=None):
    """Alg 1; gs_sweeps multicolour Gauss-Seidel sweeps with the given
    colouring smooth x~ (step 7).  Returns (x, stats dict, mask)."""
    if gs_sweeps and colour is None:
        raise ValueError("Gauss-Seidel smoothing needs a colouring")
    col = np.zeros(max(A.n, 1), np.uint8) if colour is None else np.ascontiguousarray(colour, dtype=np.uint8)
    ncol = int(col.max()) + 1 if colour is not None and A.n else 0
    p = _Params(mark_mode, thr_mode, thr_param, exp_mode, exp_rounds, alpha, grad_layers, tol,
                tol if tol_local is None else tol_local, maxit, gs_sweeps, ncol)
    s = _Stats()
    x = _f(x0).copy()
    mask = np.zeros(max(A.n, 1), np.uint8)
    lib().orc_solve_local_then_global(*A.args(), _f(b), x, C.byref(p), C.byref(s), mask, col)
    stats = {f: getattr(s, f) for f, _ in _Stats._fields_}
    return x, stats, mask[:A.n]


def heat2d_system(nx: int, ny: int, h: float, dt: float, bc_type, bc_val, kappa, Tn):
    """CSR A and b of the Picard-linearised backward-Euler heat system (Sec. 3.2)."""
    n = nx * ny
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(5 * n, np.int32)
    av = np.empty(5 * n)
    b = np.empty(n)
    nz = lib().orc_heat2d_system(nx, ny, h, dt, np.ascontiguousarray(bc_type, np.int32), _f(bc_val), _f(kappa),
                                 _f(Tn), rp, ci, av, b)
    return csr(rp, ci[:nz].copy(), av[:nz].copy()), b


def heat2d_step(nx: int, ny: int, h: float, dt: float, p: float, bc_type, bc_val, Tn, T0=None, method=1,
                mark_mode=MARK_RESIDUAL, thr_mode=THR_EPS_NORMB, thr_param=1e-10, exp_mode=EXP_PAPER, exp_rounds=1,
                alpha=1e-4, grad_layers=0, tol=1e-10, maxit=100000, picard_tol=1e-8, max_picard=100,
                gs_sweeps=0):
    """One Picard-iterated backward-Euler step of the 2D heat problem (Sec. 3.2)
    from T^{n+1,0} = T0 (default Tn).  method 0: global PCG; 1: Alg 1.
    Returns (T^{n+1}, stats dict)."""
    prm = _Params(mark_mode, thr_mode, thr_param, exp_mode, exp_rounds, alpha, grad_layers, tol, tol, maxit,
                  gs_sweeps, 2 if gs_sweeps else 0)
    T = _f(Tn if T0 is None else T0).copy()
    hs = _HeatStats()
    col = np.zeros(nx * ny, np.uint8)
    col.reshape(ny, nx)[:] = (np.add.outer(np.arange(ny), np.arange(nx)) & 1).astype(np.uint8)
    lib().orc_heat2d_step(nx, ny, h, dt, p, np.ascontiguousarray(bc_type, np.int32), _f(bc_val), _f(Tn), T,
                          method, C.byref(prm), picard_tol, max_picard, C.byref(hs), col)
    return T, {f: getattr(hs, f) for f, _ in _HeatStats._fields_}


def adjoint_grad_k_2d(nx: int, ny: int, k, x, lam) -> np.ndarray:
    """dL/dk per cell for the 2D harmonic-mean operator, given state and adjoint."""
    dk = np.empty(nx * ny)
    lib().orc_adjoint_grad_k_2d(nx, ny, _f(k), _f(x), _f(lam), dk)
    return dk


def from_stencil(op) -> CSR:
    """CSR of a gen.Stencil (convenience; the conversion itself lives in gen)."""
    from gen import stencil_to_csr
    return csr(*stencil_to_csr(op))
