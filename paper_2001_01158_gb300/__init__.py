"""GB300 library for the local character-based linear solve of Ye, An & Xu
(arXiv 2001.01158): mark a local domain from the residual (Alg 3) or the
gradient (Alg 2) of the previous iterate, extract and solve the local
subsystem (Eq. loc-equ), then finish with a warm-started global
Jacobi-preconditioned CG (Alg 1).

This module is the Python binding of the C ABI in ``include/lc_api.h``:
argument marshalling only.  Every step of the path runs in the CUDA kernels
of ``liblc.so`` (built by :func:`build`); PyTorch supplies device memory and
streams.  There is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

from .build import CHECKED_LIB, LIB, build_library

__all__ = [
    "LcError", "Context", "StencilOperator", "CsrOperator", "MarkParams", "SolveParams", "Params", "Stats",
    "Subsystem", "mark_residual", "mark_gradient", "extract", "pcg_solve", "solve_local_then_global", "build",
    "lib", "THR_EPS_NORMB", "THR_REL_MAX", "EXP_NONE", "EXP_DILATE", "EXP_PAPER", "MARK_RESIDUAL",
    "MARK_GRADIENT", "PREC_FP64", "PREC_MIXED",
]

LC_OK, LC_ERR_INVALID_ARG, LC_ERR_CUDA, LC_ERR_NO_MEMORY, LC_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
LC_ERR_BREAKDOWN, LC_ERR_TIMEOUT, LC_ERR_TOO_LARGE, LC_ERR_UNSUPPORTED = 5, 6, 7, 8
THR_EPS_NORMB, THR_REL_MAX = 0, 1
EXP_NONE, EXP_DILATE, EXP_PAPER = 0, 1, 2
MARK_RESIDUAL, MARK_GRADIENT = 0, 1
PREC_FP64, PREC_MIXED = 0, 1


class LcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lc error {code}: {msg}")
        self.code = code


class MarkParams(C.Structure):
    _fields_ = [("thr_mode", C.c_int32), ("thr_param", C.c_double), ("exp_mode", C.c_int32),
                ("exp_rounds", C.c_int32)]


class SolveParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("inner_tol", C.c_double), ("max_outer", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("mark_mode", C.c_int32), ("mark", MarkParams), ("alpha", C.c_double),
                ("grad_layers", C.c_int32), ("global_", SolveParams), ("local", SolveParams),
                ("gs_sweeps", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("n", C.c_int32), ("K", C.c_int32), ("nnzB", C.c_int32),
                ("it_local", C.c_int32), ("it_global", C.c_int32), ("early_exit", C.c_int32),
                ("restarts", C.c_int32), ("tau", C.c_double), ("eta", C.c_double),
                ("relres_tilde", C.c_double), ("relres_final", C.c_double),
                ("t_mark_ms", C.c_float), ("t_extract_ms", C.c_float), ("t_local_ms", C.c_float),
                ("t_global_ms", C.c_float), ("t_total_ms", C.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


BC_DIRICHLET, BC_NEUMANN = 0, 1


class HeatParams(C.Structure):
    _fields_ = [("h", C.c_double), ("dt", C.c_double), ("p", C.c_double), ("bc_type", C.c_int32 * 4),
                ("bc_val", C.c_double * 4), ("method", C.c_int32), ("params", Params), ("picard_tol", C.c_double),
                ("max_picard", C.c_int32)]


class HeatStats(C.Structure):
    _fields_ = [("picard_its", C.c_int32), ("it_local", C.c_int32), ("it_global", C.c_int32),
                ("K_sum", C.c_int32), ("early_exits", C.c_int32), ("status", C.c_int32),
                ("last_update", C.c_double), ("t_solve_ms", C.c_float), ("t_total_ms", C.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class _Subsys(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in ("g2l", "l2g", "rowptr", "col", "val", "rhs", "xL0", "K", "nnz")]


_lib = None


def build(force: bool = False, checked: bool = False) -> str:
    """Compile liblc.so for sm_103a (in-tree) and return its path; with
    checked=True the bounds-checked build (-DLC_CHECKED) instead."""
    return build_library(force=force, checked=checked)


def library_path() -> str:
    """The library this process loads: the bounds-checked build when the
    environment sets LC_CHECKED=1, else the ordinary one."""
    return CHECKED_LIB if os.environ.get("LC_CHECKED", "0") == "1" else LIB


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2001_01158_gb300.build() "
                           "(the library has no CPU fallback)")
    L = C.CDLL(path)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    L.lc_ctx_create.argtypes = [C.POINTER(vp), C.c_int]
    L.lc_ctx_destroy.argtypes = [vp]
    L.lc_op_create_csr.argtypes = [vp, C.POINTER(vp), i32, i64, vp, vp, vp]
    L.lc_op_create_stencil.argtypes = [vp, C.POINTER(vp), i32, C.POINTER(i32), vp, vp, vp, vp]
    L.lc_op_destroy.argtypes = [vp]
    L.lc_mark_residual.argtypes = [vp, vp, vp, vp, C.POINTER(MarkParams), vp, vp, vp, vp, vp]
    L.lc_mark_gradient.argtypes = [vp, vp, vp, d, i32, vp, vp, vp, vp]
    L.lc_extract.argtypes = [vp, vp, vp, vp, vp, C.POINTER(_Subsys), vp]
    L.lc_pcg_solve.argtypes = [vp, vp, vp, vp, C.POINTER(SolveParams), C.POINTER(Stats), vp]
    L.lc_solve_local_then_global.argtypes = [vp, vp, vp, vp, C.POINTER(Params), C.POINTER(Stats), vp]
    L.lc_error_string.argtypes = [C.c_int]
    L.lc_error_string.restype = C.c_char_p
    L.lc_last_error.argtypes = [vp]
    L.lc_last_error.restype = C.c_char_p
    L.lc_kernel_launch_count.argtypes = []
    L.lc_kernel_launch_count.restype = C.c_int64
    L.lc_op_set_tuning.argtypes = [vp, C.c_char_p, i32]
    L.lc_op_get_tuning.argtypes = [vp, C.c_char_p, C.POINTER(i32)]
    L.lc_assemble_diffusion_2d.argtypes = [vp, C.POINTER(i32), vp, d, vp, vp, vp, vp]
    L.lc_op_refresh.argtypes = [vp, vp]
    L.lc_adjoint_grad_k_2d.argtypes = [vp, C.POINTER(i32), vp, vp, vp, vp, vp]
    L.lc_gs_smooth.argtypes = [vp, vp, vp, vp, i32, vp]
    L.lc_op_dot.argtypes = [vp, vp, vp, vp, vp, vp]
    L.lc_selftest_barrier_timeout.argtypes = [vp, vp, i32, d, C.POINTER(i32)]
    L.lc_heat2d_assemble.argtypes = [vp, C.POINTER(i32), d, d, C.POINTER(i32), C.POINTER(d), vp, vp, vp, vp, vp,
                                     vp, vp]
    L.lc_heat2d_step.argtypes = [vp, vp, C.POINTER(HeatParams), vp, vp, vp, vp, vp, vp, vp, C.POINTER(HeatStats), vp]
    L.lc_op_set_colouring.argtypes = [vp, vp, i32]
    L.lc_checked_status.argtypes = [C.POINTER(i32), C.c_char_p, i32]
    L.lc_checked_selftest.argtypes = [vp]
    _lib = L
    return L


def _ptr(t: torch.Tensor | None, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """lc_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = device
        h = C.c_void_p()
        rc = lib().lc_ctx_create(C.byref(h), device)
        if rc:
            raise LcError(rc, lib().lc_error_string(rc).decode())
        self.h = h

    def check(self, rc: int, allow=()):
        if rc and rc not in allow:
            raise LcError(rc, f"{lib().lc_error_string(rc).decode()}: {lib().lc_last_error(self.h).decode()}")
        return rc

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lc_ctx_destroy(self.h)
            self.h = None


class _Operator:
    n: int
    nnz: int

    def set_colouring(self, colour, ncolours: int | None = None):
        """lc_op_set_colouring: uint8 device colours of a CSR operator's rows
        for Gauss-Seidel (None removes; stencil operators refuse it)."""
        if colour is None:
            self._colour = None
            return self.ctx.check(lib().lc_op_set_colouring(self.h, None, 0))
        if ncolours is None:
            ncolours = int(colour.max().item()) + 1
        self._colour = colour
        return self.ctx.check(lib().lc_op_set_colouring(self.h, _ptr(colour, torch.uint8, "colour"), int(ncolours)))

    def set_tuning(self, key: str, value: int):
        """lc_op_set_tuning (launch-shape knobs for the autotuner)."""
        return self.ctx.check(lib().lc_op_set_tuning(self.h, key.encode(), int(value)))

    def get_tuning(self, key: str) -> int:
        v = C.c_int32()
        self.ctx.check(lib().lc_op_get_tuning(self.h, key.encode(), C.byref(v)))
        return v.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lc_op_destroy(self.h)
            self.h = None


class StencilOperator(_Operator):
    """5-point (2D) or 7-point (3D) operator from device arrays D, Tx, Ty(, Tz)."""

    def __init__(self, ctx: Context, shape, D, Tx, Ty, Tz=None):
        nx, ny, nz = (tuple(shape) + (1,))[:3]
        self.ctx, self.shape = ctx, (int(nx), int(ny), int(nz))
        self.dim = 3 if Tz is not None else 2
        self._keep = (D, Tx, Ty, Tz)
        self.n = nx * ny * nz
        self.nnz = self.n + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1))
        for name, t in (("D", D), ("Tx", Tx), ("Ty", Ty), ("Tz", Tz)):
            if t is not None and t.numel() != self.n:
                raise ValueError(f"{name} has {t.numel()} values, expected {self.n}")
        sh = (C.c_int32 * 3)(nx, ny, nz)
        h = C.c_void_p()
        ctx.check(lib().lc_op_create_stencil(ctx.h, C.byref(h), self.dim, sh, _ptr(D, torch.float64, "D"),
                                             _ptr(Tx, torch.float64, "Tx"), _ptr(Ty, torch.float64, "Ty"),
                                             _ptr(Tz, torch.float64, "Tz")))
        self.h = h


class CsrOperator(_Operator):
    """General sparse operator from device CSR arrays (int32, int32, float64)."""

    def __init__(self, ctx: Context, rowptr, col, val):
        self.ctx = ctx
        self._keep = (rowptr, col, val)
        self.n = rowptr.numel() - 1
        self.nnz = col.numel()
        h = C.c_void_p()
        ctx.check(lib().lc_op_create_csr(ctx.h, C.byref(h), self.n, self.nnz, _ptr(rowptr, torch.int32, "rowptr"),
                                         _ptr(col, torch.int32, "col"), _ptr(val, torch.float64, "val")))
        self.h = h


@dataclass
class Subsystem:
    """Caller-allocated outputs of extract() (device tensors of full capacity)."""
    g2l: torch.Tensor
    l2g: torch.Tensor
    rowptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor
    rhs: torch.Tensor
    xL0: torch.Tensor
    K: torch.Tensor
    nnz: torch.Tensor

    @staticmethod
    def empty(op: _Operator, device=None) -> "Subsystem":
        dev = device or torch.device("cuda", op.ctx.device)
        n, nnz = op.n, op.nnz
        return Subsystem(torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
                         torch.empty(n + 1, dtype=torch.int32, device=dev),
                         torch.empty(max(nnz, 1), dtype=torch.int32, device=dev),
                         torch.empty(max(nnz, 1), dtype=torch.float64, device=dev),
                         torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.float64, device=dev),
                         torch.zeros(1, dtype=torch.int32, device=dev), torch.zeros(1, dtype=torch.int32, device=dev))

    def trimmed(self) -> dict:
        """Host copies of the meaningful parts (synchronises)."""
        K, nz = int(self.K.item()), int(self.nnz.item())
        return {"K": K, "nnz": nz, "g2l": self.g2l.cpu().numpy(), "l2g": self.l2g[:K].cpu().numpy(),
                "rowptr": self.rowptr[:K + 1].cpu().numpy(), "col": self.col[:nz].cpu().numpy(),
                "val": self.val[:nz].cpu().numpy(), "rhs": self.rhs[:K].cpu().numpy(),
                "xL0": self.xL0[:K].cpu().numpy()}


def mark_residual(ctx: Context, op: _Operator, b, x0, params: MarkParams, mask, K, r0=None, tau=None, stream=None):
    """lc_mark_residual: mask (uint8[N]), K (int32[1]), optional r0 (float64[N]) and tau (float64[1])."""
    return ctx.check(lib().lc_mark_residual(ctx.h, op.h, _ptr(b, torch.float64, "b"), _ptr(x0, torch.float64, "x0"),
                                            C.byref(params), _ptr(mask, torch.uint8, "mask"),
                                            _ptr(r0, torch.float64, "r0"), _ptr(K, torch.int32, "K"),
                                            _ptr(tau, torch.float64, "tau"), _stream(stream)))


def heat2d_assemble(ctx: Context, shape, h: float, dt: float, bc_type, bc_val, kappa, Tn, D, Tx, Ty, b,
                    stream=None):
    """lc_heat2d_assemble: the Picard-linearised heat system (Sec. 3.2) as stencil arrays and b."""
    sh = (C.c_int32 * 2)(*shape[:2])
    return ctx.check(lib().lc_heat2d_assemble(ctx.h, sh, float(h), float(dt), (C.c_int32 * 4)(*bc_type),
                                              (C.c_double * 4)(*bc_val), _ptr(kappa, torch.float64, "kappa"),
                                              _ptr(Tn, torch.float64, "Tn"), _ptr(D, torch.float64, "D"),
                                              _ptr(Tx, torch.float64, "Tx"), _ptr(Ty, torch.float64, "Ty"),
                                              _ptr(b, torch.float64, "b"), _stream(stream)))


def heat_params(h: float, dt: float, p: float, bc_type, bc_val, method: int = 1, params: "Params | None" = None,
                picard_tol: float = 1e-8, max_picard: int = 100) -> HeatParams:
    """lc_heat2d_params; params defaults to Alg 1 with the paper's residual
    marking (eps ||b|| / sqrt(N) with eps = 1e-10, E_max = 1) at tolerance 1e-10."""
    if params is None:
        params = default_params(MARK_RESIDUAL, THR_EPS_NORMB, 1e-10, EXP_PAPER, 1, tol=1e-10)
    return HeatParams(h, dt, p, (C.c_int32 * 4)(*bc_type), (C.c_double * 4)(*bc_val), method, params, picard_tol,
                      max_picard)


def heat2d_step(ctx: Context, op: "StencilOperator", hp: HeatParams, Tn, T, D, Tx, Ty, b, work,
                stats: HeatStats | None = None, stream=None) -> HeatStats:
    """lc_heat2d_step: one Picard-iterated backward-Euler step (T in: T^{n+1,0}, out: T^{n+1})."""
    st = stats if stats is not None else HeatStats()
    ctx.check(lib().lc_heat2d_step(ctx.h, op.h, C.byref(hp), _ptr(Tn, torch.float64, "Tn"),
                                   _ptr(T, torch.float64, "T"), _ptr(D, torch.float64, "D"),
                                   _ptr(Tx, torch.float64, "Tx"), _ptr(Ty, torch.float64, "Ty"),
                                   _ptr(b, torch.float64, "b"), _ptr(work, torch.float64, "work"), C.byref(st),
                                   _stream(stream)))
    return st


def selftest_barrier_timeout(ctx: Context, op: _Operator, blocks: int, limit_ms: float) -> int:
    """lc_selftest_barrier_timeout: the status a barrier that cannot complete records."""
    st = C.c_int32()
    ctx.check(lib().lc_selftest_barrier_timeout(ctx.h, op.h, int(blocks), float(limit_ms), C.byref(st)))
    return st.value


def dot(ctx: Context, op: _Operator, x, y, out, stream=None):
    """lc_op_dot: reproducible FP64 dot product into the device scalar `out`."""
    return ctx.check(lib().lc_op_dot(ctx.h, op.h, _ptr(x, torch.float64, "x"), _ptr(y, torch.float64, "y"),
                                     _ptr(out, torch.float64, "out"), _stream(stream)))


def gs_smooth(ctx: Context, op: _Operator, b, x, sweeps: int, stream=None):
    """lc_gs_smooth: multicolour Gauss-Seidel sweeps on A x = b, in place in x."""
    return ctx.check(lib().lc_gs_smooth(ctx.h, op.h, _ptr(b, torch.float64, "b"), _ptr(x, torch.float64, "x"),
                                        int(sweeps), _stream(stream)))


def mark_gradient(ctx: Context, op: _Operator, x0, alpha: float, layers: int, mask, K, gmax=None, stream=None):
    """lc_mark_gradient."""
    return ctx.check(lib().lc_mark_gradient(ctx.h, op.h, _ptr(x0, torch.float64, "x0"), float(alpha), int(layers),
                                            _ptr(mask, torch.uint8, "mask"), _ptr(K, torch.int32, "K"),
                                            _ptr(gmax, torch.float64, "gmax"), _stream(stream)))


def extract(ctx: Context, op: _Operator, mask, b, x0, out: Subsystem, stream=None):
    """lc_extract into caller-allocated `out`."""
    s = _Subsys(*(_ptr(getattr(out, f), None, f) for f, _ in _Subsys._fields_))
    return ctx.check(lib().lc_extract(ctx.h, op.h, _ptr(mask, torch.uint8, "mask"), _ptr(b, torch.float64, "b"),
                                      _ptr(x0, torch.float64, "x0"), C.byref(s), _stream(stream)))


def pcg_solve(ctx: Context, op: _Operator, b, x, params: SolveParams, stats: Stats | None = None, stream=None,
              allow_not_converged=False):
    """lc_pcg_solve: x holds x0 on entry and the solution on return."""
    allow = (LC_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    return ctx.check(lib().lc_pcg_solve(ctx.h, op.h, _ptr(b, torch.float64, "b"), _ptr(x, torch.float64, "x"),
                                        C.byref(params), C.byref(stats) if stats is not None else None,
                                        _stream(stream)), allow)


def solve_local_then_global(ctx: Context, op: _Operator, b, x, params: Params, stats: Stats | None = None,
                            stream=None, allow_not_converged=False):
    """lc_solve_local_then_global (Alg 1): x holds x0 on entry and the solution on return."""
    allow = (LC_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    return ctx.check(lib().lc_solve_local_then_global(ctx.h, op.h, _ptr(b, torch.float64, "b"),
                                                      _ptr(x, torch.float64, "x"), C.byref(params),
                                                      C.byref(stats) if stats is not None else None,
                                                      _stream(stream)), allow)


def adjoint_grad(ctx: Context, op: "StencilOperator", k, dt: float, x, gx, lam, dk, params: Params,
                 stats: Stats | None = None, stream=None):
    """lc_adjoint_grad: re-assembles A(k) into op's arrays, solves A lam = gx by
    Alg 1 (lam: start in, dL/db out) and writes dL/dk into dk."""
    L = lib()
    vp = C.c_void_p
    L.lc_adjoint_grad.argtypes = [vp, vp, vp, C.c_double, vp, vp, vp, vp, C.POINTER(Params), C.POINTER(Stats), vp]
    return ctx.check(L.lc_adjoint_grad(ctx.h, op.h, _ptr(k, torch.float64, "k"), float(dt),
                                       _ptr(x, torch.float64, "x"), _ptr(gx, torch.float64, "gx"),
                                       _ptr(lam, torch.float64, "lam"), _ptr(dk, torch.float64, "dk"),
                                       C.byref(params), C.byref(stats) if stats is not None else None,
                                       _stream(stream)))


def kernel_launch_count() -> int:
    """Kernels this library has launched in this process (lc_kernel_launch_count)."""
    return int(lib().lc_kernel_launch_count())


def checked_selftest(stream=None) -> None:
    """Record one deliberate, harmless index-check failure (lc_checked_selftest);
    raises LcError with LC_ERR_UNSUPPORTED in an ordinary build."""
    rc = lib().lc_checked_selftest(_stream(stream))
    if rc:
        raise LcError(rc, lib().lc_error_string(rc).decode())


def checked_status() -> tuple[int, str]:
    """(number of kernel files with a failed index check, "file:line" of the
    first) from the bounds-checked build, clearing the records
    (lc_checked_status; synchronise the device first).  Raises LcError with
    LC_ERR_UNSUPPORTED when the loaded library is the ordinary build."""
    n = C.c_int32(0)
    buf = C.create_string_buffer(256)
    rc = lib().lc_checked_status(C.byref(n), buf, len(buf))
    if rc:
        raise LcError(rc, buf.value.decode())
    return int(n.value), buf.value.decode()


def default_params(mark_mode=MARK_RESIDUAL, thr_mode=THR_REL_MAX, thr_param=1e-3, exp_mode=EXP_DILATE, exp_rounds=2,
                   alpha=1e-3, grad_layers=2, tol=1e-8, tol_local=None, max_iter=100000,
                   precision=PREC_FP64, inner_tol=1e-5, max_outer=30, gs_sweeps=0) -> Params:
    """Alg 1 parameters with the relative-threshold, 2-layer defaults."""
    g = SolveParams(tol, max_iter, precision, inner_tol, max_outer)
    l = SolveParams(tol if tol_local is None else tol_local, max_iter, precision, inner_tol, max_outer)
    return Params(mark_mode, MarkParams(thr_mode, thr_param, exp_mode, exp_rounds), alpha, grad_layers, g, l,
                  gs_sweeps)


LC_NOALLOC_MAX_CELLS = 4194304


def mark_residual_stencil_noalloc(shape, D, Tx, Ty, Tz, b, x0, params: MarkParams, mask, r0, K, tau=None,
                                  stream=None) -> int:
    """lc_mark_residual_stencil_noalloc: residual marking for callers that
    cannot allocate device memory (no context, no operator).  Scratch lives in
    a fixed device array inside the library, so grids are limited to
    LC_NOALLOC_MAX_CELLS cells and calls must not overlap on the GPU.
    Raises LcError on a non-zero return code."""
    L = lib()
    f = L.lc_mark_residual_stencil_noalloc
    vp = C.c_void_p
    f.argtypes = [C.c_int32, C.POINTER(C.c_int32), vp, vp, vp, vp, vp, vp, C.POINTER(MarkParams), vp, vp, vp, vp,
                  vp]
    nx, ny, nz = (tuple(shape) + (1,))[:3]
    # a 3D grid needs its z faces: without Tz the C side would mark only the
    # first nx*ny cells of buffers that hold nx*ny*nz
    if Tz is None and nz > 1:
        raise ValueError(f"shape {tuple(shape)} has nz = {nz} > 1 but Tz is None")
    dim = 3 if Tz is not None else 2
    sh = (C.c_int32 * 3)(nx, ny, nz)
    rc = f(dim, sh, _ptr(D, torch.float64, "D"), _ptr(Tx, torch.float64, "Tx"), _ptr(Ty, torch.float64, "Ty"),
           _ptr(Tz, torch.float64, "Tz"), _ptr(b, torch.float64, "b"), _ptr(x0, torch.float64, "x0"),
           C.byref(params), _ptr(mask, torch.uint8, "mask"), _ptr(r0, torch.float64, "r0"),
           _ptr(K, torch.int32, "K"), _ptr(tau, torch.float64, "tau"), _stream(stream))
    if rc:
        extra = f" (grid of {nx * ny * nz} cells exceeds LC_NOALLOC_MAX_CELLS = {LC_NOALLOC_MAX_CELLS})" \
            if rc == LC_ERR_TOO_LARGE else ""
        raise LcError(rc, L.lc_error_string(rc).decode() + extra)
    return rc


class Batch:
    """lc_batch: many independent 2D systems solved by Alg 1 in one launch.

    `systems` is a list of (nx, ny, D, Tx, Ty) with device FP64 arrays; they
    are concatenated into one set of coefficient arrays owned by this object."""

    def __init__(self, ctx: Context, systems):
        L = lib()
        vp, i32 = C.c_void_p, C.c_int32
        L.lc_batch_create.argtypes = [vp, C.POINTER(vp), i32, C.POINTER(i32), C.POINTER(i32), vp, vp, vp]
        L.lc_batch_destroy.argtypes = [vp]
        L.lc_batch_solve.argtypes = [vp, vp, vp, vp, C.POINTER(Params), vp]
        L.lc_batch_capture.argtypes = [vp, vp, vp, vp, C.POINTER(Params)]
        L.lc_batch_replay.argtypes = [vp, vp]
        L.lc_batch_stats.argtypes = [vp, C.POINTER(Stats), vp]
        L.lc_batch_set_tuning.argtypes = [vp, C.c_char_p, i32]
        self.ctx = ctx
        self.nx = [int(s[0]) for s in systems]
        self.ny = [int(s[1]) for s in systems]
        self.sizes = [a * b for a, b in zip(self.nx, self.ny)]
        self.offsets = [0]
        for n in self.sizes:
            self.offsets.append(self.offsets[-1] + n)
        self.cells = self.offsets[-1]
        self.D = torch.cat([s[2].reshape(-1) for s in systems]).contiguous()
        self.Tx = torch.cat([s[3].reshape(-1) for s in systems]).contiguous()
        self.Ty = torch.cat([s[4].reshape(-1) for s in systems]).contiguous()
        torch.cuda.current_stream().synchronize()
        nsys = len(systems)
        h = C.c_void_p()
        ctx.check(L.lc_batch_create(ctx.h, C.byref(h), nsys, (i32 * nsys)(*self.nx), (i32 * nsys)(*self.ny),
                                    _ptr(self.D, torch.float64, "D"), _ptr(self.Tx, torch.float64, "Tx"),
                                    _ptr(self.Ty, torch.float64, "Ty")))
        self.h = h
        self.nsys = nsys

    def solve(self, b, x, params: Params, stream=None):
        return self.ctx.check(lib().lc_batch_solve(self.ctx.h, self.h, _ptr(b, torch.float64, "b"),
                                                   _ptr(x, torch.float64, "x"), C.byref(params), _stream(stream)))

    def capture(self, b, x, params: Params):
        """Capture the batched solve for these b, x, params into a CUDA graph."""
        self._captured = (b, x)
        return self.ctx.check(lib().lc_batch_capture(self.ctx.h, self.h, _ptr(b, torch.float64, "b"),
                                                     _ptr(x, torch.float64, "x"), C.byref(params)))

    def replay(self, stream=None):
        return self.ctx.check(lib().lc_batch_replay(self.h, _stream(stream)))

    def stats(self, stream=None, allow_not_converged=False):
        st = (Stats * self.nsys)()
        allow = (LC_ERR_NOT_CONVERGED, LC_ERR_BREAKDOWN) if allow_not_converged else ()
        self.ctx.check(lib().lc_batch_stats(self.h, st, _stream(stream)), allow)
        return [s.as_dict() for s in st]

    def domain(self, sys: int, stream=None) -> dict:
        """lc_batch_domain: system `sys`'s final mask and local subsystem
        (g2l, l2g, rowptr, col, val, rhs) from the last solve, as CPU numpy
        arrays."""
        st = self.stats(stream, allow_not_converged=True)[sys]
        n, K, nz = self.sizes[sys], st["K"], st["nnzB"]
        dev = self.D.device
        out = {"mask": torch.empty(n, dtype=torch.uint8, device=dev),
               "g2l": torch.empty(n, dtype=torch.int32, device=dev),
               "l2g": torch.empty(max(K, 1), dtype=torch.int32, device=dev),
               "rowptr": torch.empty(K + 1, dtype=torch.int32, device=dev),
               "col": torch.empty(max(nz, 1), dtype=torch.int32, device=dev),
               "val": torch.empty(max(nz, 1), dtype=torch.float64, device=dev),
               "rhs": torch.empty(max(K, 1), dtype=torch.float64, device=dev)}
        L = lib()
        L.lc_batch_domain.argtypes = [C.c_void_p, C.c_int32] + [C.c_void_p] * 8
        self.ctx.check(L.lc_batch_domain(self.h, sys, *[out[k].data_ptr() for k in
                                                        ("mask", "g2l", "l2g", "rowptr", "col", "val", "rhs")],
                                         _stream(stream)))
        torch.cuda.synchronize(dev)
        res = {k: v.cpu().numpy() for k, v in out.items()}
        res["l2g"], res["rhs"] = res["l2g"][:K], res["rhs"][:K]
        res["col"], res["val"] = res["col"][:nz], res["val"][:nz]
        return res

    def set_tuning(self, key: str, value: int):
        return self.ctx.check(lib().lc_batch_set_tuning(self.h, key.encode(), int(value)))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lc_batch_destroy(self.h)
            self.h = None


def batch_params(beta=1e-3, layers=2, tol=1e-8, tol_local=None, inner_tol=1e-4, max_outer=30,
                 max_inner=20000) -> Params:
    """Parameters accepted by the batched solve (relative threshold, layer
    dilation, mixed precision)."""
    return default_params(MARK_RESIDUAL, THR_REL_MAX, beta, EXP_DILATE if layers else EXP_NONE, layers, tol=tol,
                          tol_local=tol_local, max_iter=max_inner, precision=PREC_MIXED, inner_tol=inner_tol,
                          max_outer=max_outer)
