"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (the operators' default tuning):

- 2048 x 2048 moving front (the bench workload), a system of the sequence's
  form b = x0/dt + s^1 with x0 = s^0: residual marking (the relative
  threshold with 2 layers, and the paper's Alg 3 marking of the bench's
  headline), the subsystem and the whole of Alg 1 against the oracle (masks
  and subsystem bit for bit, the solution within 1e-9, relres by the
  oracle); gradient marking bit for bit.
- 256^3 anisotropic 3D: marking and subsystem bit for bit; the FP64 and the
  mixed-precision solves to relres 1e-10, evaluated by the oracle, and both
  solutions against the oracle's own serial FP64 Jacobi-PCG solution of the
  16.7 M unknowns (FP64 within 1e-9, mixed precision within 1e-7).
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2001_01158_gb300 as lcg

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def ctx():
    lcg.build()
    return lcg.Context(0)


def cu(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def stencil_op(ctx, op):
    return lcg.StencilOperator(ctx, op.shape, cu(op.D), cu(op.Tx), cu(op.Ty), cu(op.Tz) if op.Tz is not None else None)


@pytest.fixture(scope="module")
def front2048():
    d = gen.cfg2_fronts2d(seed=0, n=2048)
    x0 = d["seq"].source(0)
    b = x0 / d["op"].meta["dt"] + d["seq"].source(1)
    return d["op"], oracle.from_stencil(d["op"]), b, x0


def check_mark_and_extract(ctx, gop, A, b, x0, case):
    n = A.n
    ref = oracle.mark_residual(A, b, x0, *case)
    mask = torch.empty(n, dtype=torch.uint8, device=DEV)
    r0 = torch.empty(n, dtype=torch.float64, device=DEV)
    K = torch.zeros(1, dtype=torch.int32, device=DEV)
    tau = torch.zeros(1, dtype=torch.float64, device=DEV)
    lcg.mark_residual(ctx, gop, cu(b), cu(x0), lcg.MarkParams(*case), mask, K, r0, tau)
    torch.cuda.synchronize()
    m = mask.cpu().numpy()
    assert np.array_equal(m, ref["mask"]) and int(K.item()) == ref["K"] > 0
    assert bits([tau.item()])[0] == bits([ref["tau"]])[0]
    assert np.array_equal(bits(r0.cpu().numpy()), bits(ref["r"]))
    e = oracle.extract(A, m, b, x0)
    out = lcg.Subsystem.empty(gop)
    lcg.extract(ctx, gop, mask, cu(b), cu(x0), out)
    torch.cuda.synchronize()
    got = out.trimmed()
    assert got["K"] == e["K"] and np.array_equal(got["l2g"], e["l2g"])
    assert np.array_equal(got["rowptr"], e["B"].rowptr) and np.array_equal(got["col"], e["B"].col)
    assert np.array_equal(bits(got["val"]), bits(e["B"].val)) and np.array_equal(bits(got["rhs"]), bits(e["rhs"]))
    return ref["K"]


def test_front2048_marking_extraction_and_alg1(ctx, front2048):
    op, A, b, x0 = front2048
    gop = stencil_op(ctx, op)
    K = check_mark_and_extract(ctx, gop, A, b, x0, (lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2))
    xr, sr, _ = oracle.solve_local_then_global(A, b, x0, tol=1e-8)
    prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2, tol=1e-8)
    x = cu(x0)
    st = lcg.Stats()
    lcg.solve_local_then_global(ctx, gop, cu(b), x, prm, st)
    xg = x.cpu().numpy()
    assert st.K == sr["K"] == K and st.nnzB == sr["nnzB"]
    assert abs(st.it_local - sr["it_local"]) <= 1 and abs(st.it_global - sr["it_global"]) <= 1
    assert st.relres_tilde == pytest.approx(sr["relres_tilde"], rel=1e-6)
    assert oracle.relres(A, b, xg) <= 1e-8
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)


def test_front2048_paper_marking_alg1(ctx, front2048):
    """The bench's headline setting: residual marking as the paper runs it
    (tau = eps ||b|| / sqrt(N), eps = 1e-8, Alg 3 with E_max = 1), the
    default (pipelined) local solve, against the oracle's Alg 1."""
    op, A, b, x0 = front2048
    gop = stencil_op(ctx, op)
    case = (lcg.THR_EPS_NORMB, 1e-8, lcg.EXP_PAPER, 1)
    K = check_mark_and_extract(ctx, gop, A, b, x0, case)
    xr, sr, _ = oracle.solve_local_then_global(A, b, x0, thr_mode=oracle.THR_EPS_NORMB, thr_param=1e-8,
                                               exp_mode=oracle.EXP_PAPER, exp_rounds=1, tol=1e-8)
    prm = lcg.default_params(lcg.MARK_RESIDUAL, *case, tol=1e-8)
    assert gop.get_tuning("local_pipelined") == 1
    x = cu(x0)
    st = lcg.Stats()
    lcg.solve_local_then_global(ctx, gop, cu(b), x, prm, st)
    xg = x.cpu().numpy()
    assert st.K == sr["K"] == K and st.nnzB == sr["nnzB"]
    assert abs(st.it_local - sr["it_local"]) <= 1 and abs(st.it_global - sr["it_global"]) <= 1
    assert st.early_exit == sr["early_exit"]
    assert oracle.relres(A, b, xg) <= 1e-8
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)


def test_front2048_gradient_marking(ctx, front2048):
    op, A, b, x0 = front2048
    ref = oracle.mark_gradient(A, x0, 1e-3, 2)
    mask = torch.empty(A.n, dtype=torch.uint8, device=DEV)
    K = torch.zeros(1, dtype=torch.int32, device=DEV)
    gmax = torch.zeros(1, dtype=torch.float64, device=DEV)
    lcg.mark_gradient(ctx, stencil_op(ctx, op), cu(x0), 1e-3, 2, mask, K, gmax)
    torch.cuda.synchronize()
    assert np.array_equal(mask.cpu().numpy(), ref["mask"]) and int(K.item()) == ref["K"] > 0
    assert bits([gmax.item()])[0] == bits([ref["gmax"]])[0]


def test_aniso256_marking_and_solves(ctx):
    d = gen.cfg3_aniso3d(seed=0, n=256)
    op = d["op"]
    A = oracle.from_stencil(op)
    gop = stencil_op(ctx, op)
    check_mark_and_extract(ctx, gop, A, d["b"], d["x0"], (lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2))
    b = cu(d["b"])
    x64 = cu(d["x0"])
    st = lcg.Stats()
    lcg.pcg_solve(ctx, gop, b, x64, lcg.SolveParams(1e-10, 200000, lcg.PREC_FP64, 0.0, 0), st)
    xm = cu(d["x0"])
    stm = lcg.Stats()
    prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2, tol=1e-10,
                             precision=lcg.PREC_MIXED, inner_tol=1e-5)
    lcg.solve_local_then_global(ctx, gop, b, xm, prm, stm)
    x64h, xmh = x64.cpu().numpy(), xm.cpu().numpy()
    assert oracle.relres(A, d["b"], x64h) <= 1e-10
    assert oracle.relres(A, d["b"], xmh) <= 1e-10
    # against the oracle's own FP64 Jacobi-PCG solution (serial, same
    # tolerance): the FP64 solve runs the same algorithm, so it tracks the
    # oracle's iterates (1e-9); the mixed-precision Alg 1 result meets the
    # same residual by another path, its error is bounded by the conditioning
    xo, so, _, _ = oracle.pcg(A, d["b"], d["x0"], tol=1e-10)
    assert so == oracle.OK
    no = np.linalg.norm(xo)
    e64, em = np.linalg.norm(x64h - xo) / no, np.linalg.norm(xmh - xo) / no
    assert e64 <= 1e-9, e64
    assert em <= 1e-7, em
