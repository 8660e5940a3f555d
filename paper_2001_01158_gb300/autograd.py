"""Differentiable 2D diffusion solve: x = A(k)^-1 b by the local
character-based method, with gradients with respect to the per-cell
conductivity k and the right-hand side b.

Forward: assemble A(k) on the GPU (lc_assemble_diffusion_2d), refresh the
operator's derived data, solve by Alg 1 (lc_solve_local_then_global).  Only
k and x are saved.  Backward: one lc_adjoint_grad call, which re-assembles
A(k) (recomputed, not stored: no Krylov state is kept from the forward),
solves the adjoint A lambda = dL/dx on the same local-then-global path (A is
symmetric) and forms dL/db = lambda and dL/dk with the adjoint kernel.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import (Context, Params, StencilOperator, Stats, _ptr, _stream, adjoint_grad, default_params, lib,
               solve_local_then_global)

__all__ = ["DiffusionSolve", "diffusion_solve"]

_contexts: dict = {}
_operators: dict = {}


def _context(device: int) -> Context:
    if device not in _contexts:
        _contexts[device] = Context(device)
    return _contexts[device]


class _Assembled:
    """D, Tx, Ty buffers of one grid shape and the operator built on them."""

    def __init__(self, ctx: Context, ny: int, nx: int, device):
        n = nx * ny
        self.shape = (nx, ny)
        self.D = torch.empty(n, dtype=torch.float64, device=device)
        self.Tx = torch.empty(n, dtype=torch.float64, device=device)
        self.Ty = torch.empty(n, dtype=torch.float64, device=device)
        self.ready = False
        self.ctx = ctx
        self.op = None

    def assemble(self, k: torch.Tensor, dt: float):
        sh = (C.c_int32 * 2)(*self.shape)
        self.ctx.check(lib().lc_assemble_diffusion_2d(self.ctx.h, sh, _ptr(k, torch.float64, "k"), float(dt),
                                                      _ptr(self.D), _ptr(self.Tx), _ptr(self.Ty), _stream(None)))
        if self.op is None:
            torch.cuda.current_stream().synchronize()
            self.op = StencilOperator(self.ctx, (self.shape[0], self.shape[1], 1), self.D, self.Tx, self.Ty)
        else:
            self.ctx.check(lib().lc_op_refresh(self.op.h, _stream(None)))
        return self.op


def _assembled(k: torch.Tensor) -> _Assembled:
    dev = k.device.index if k.device.index is not None else torch.cuda.current_device()
    ny, nx = k.shape
    key = (dev, ny, nx)
    if key not in _operators:
        _operators[key] = _Assembled(_context(dev), ny, nx, k.device)
    return _operators[key]


class DiffusionSolve(torch.autograd.Function):
    """x = A(k)^-1 b (2D, k and b of shape (ny, nx), float64, CUDA)."""

    @staticmethod
    def forward(ctx, k, b, x0, params: Params, dt: float):
        if k.dim() != 2 or b.shape != k.shape:
            raise ValueError("k and b must be (ny, nx) tensors of the same shape")
        k = k.detach().contiguous()
        a = _assembled(k)
        op = a.assemble(k, dt)
        x = (x0.detach().clone() if x0 is not None else torch.zeros_like(b)).contiguous().view(-1)
        st = Stats()
        solve_local_then_global(a.ctx, op, b.detach().contiguous().view(-1), x, params, st)
        ctx.save_for_backward(k, x)
        ctx.params, ctx.dt = params, dt
        ctx.forward_stats = st.as_dict()
        return x.view_as(b)

    @staticmethod
    def backward(ctx, gx):
        k, x = ctx.saved_tensors
        a = _assembled(k)
        if a.op is None:
            a.assemble(k, ctx.dt)
        g = gx.detach().contiguous().view(-1)
        lam = torch.zeros_like(g)
        dk = torch.empty_like(lam)
        st = Stats()
        adjoint_grad(a.ctx, a.op, k, ctx.dt, x, g, lam, dk, ctx.params, st)   # A(k) recomputed inside
        ctx.adjoint_stats = st.as_dict()
        return dk.view_as(k), lam.view_as(k), None, None, None


def diffusion_solve(k: torch.Tensor, b: torch.Tensor, x0: torch.Tensor | None = None, params: Params | None = None,
                    dt: float = 1.0) -> torch.Tensor:
    """Differentiable x = A(k)^-1 b; params default to residual marking and
    Jacobi-PCG to relres 1e-10 for both the forward and the adjoint solve."""
    if params is None:
        params = default_params(tol=1e-10)
    return DiffusionSolve.apply(k, b, x0, params, dt)
