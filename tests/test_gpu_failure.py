"""Failure detection on the GPU without a fault.  A grid barrier that cannot
complete (one arrival more than there are blocks) gives up after its short
limit, every block records LC_ERR_TIMEOUT and returns, the host reads the
status, and the context keeps working (a solve right after matches the
oracle).  Krylov breakdown on host-made inputs (NaN in b, an indefinite
operator) is reported as LC_ERR_BREAKDOWN, as the oracle reports it."""
import time

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2001_01158_gb300 as lcg

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def test_barrier_timeout_is_reported_and_context_survives():
    lcg.build()
    ctx = lcg.Context(0)
    op = gen.random_stencil_2d(2, 64, 48)
    cu = lambda a: torch.as_tensor(a, dtype=torch.float64, device=DEV)  # noqa: E731
    gop = lcg.StencilOperator(ctx, op.shape, cu(op.D), cu(op.Tx), cu(op.Ty))
    for blocks in (1, 8, 152):
        t = time.perf_counter()
        st = lcg.selftest_barrier_timeout(ctx, gop, blocks, 50.0)
        dt = time.perf_counter() - t
        assert st == lcg.LC_ERR_TIMEOUT
        assert dt < 5.0
    # the context and the operator still work
    A = oracle.from_stencil(op)
    b = np.random.default_rng(0).standard_normal(op.n)
    x = cu(np.zeros(op.n))
    s = lcg.Stats()
    lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(1e-8, 10000, lcg.PREC_FP64, 0.0, 0), s)
    assert s.status == 0 and oracle.relres(A, b, x.cpu().numpy()) <= 1e-8
    with pytest.raises(lcg.LcError):
        lcg.selftest_barrier_timeout(ctx, gop, 4, 5000.0)   # limit above 2 s refused


def _indefinite(op):
    """The same stencil with its diagonal shrunk to 0.3 x the sum of the
    row's face conductances: positive diagonal, symmetric, indefinite."""
    import copy
    A = oracle.from_stencil(op)
    Ad = A.dense()
    off = np.abs(Ad).sum(1) - np.abs(np.diag(Ad))
    op2 = copy.copy(op)
    op2.D = 0.3 * off
    return op2


@pytest.mark.parametrize("kind", ["stencil", "csr"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_krylov_breakdown_is_reported_and_context_survives(kind, precision):
    """Krylov breakdown (p^T A p <= 0 or not finite) on host-made inputs: a NaN
    in b, and an indefinite operator with a positive diagonal.  The oracle's
    Jacobi-PCG breaks down on both (checked first); lc_pcg_solve and
    lc_solve_local_then_global return LC_ERR_BREAKDOWN, and a solve on the
    same context right after is correct."""
    lcg.build()
    ctx = lcg.Context(0)
    cu = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)  # noqa: E731
    op = gen.random_stencil_2d(5, 40, 30)
    bad = _indefinite(op)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(op.n)
    b_nan = b.copy()
    b_nan[17] = np.nan

    def make(o):
        if kind == "stencil":
            return lcg.StencilOperator(ctx, o.shape, cu(o.D), cu(o.Tx), cu(o.Ty))
        A = oracle.from_stencil(o)
        return lcg.CsrOperator(ctx, cu(A.rowptr, torch.int32), cu(A.col, torch.int32), cu(A.val))

    good_op, bad_op = make(op), make(bad)
    prec = lcg.PREC_FP64 if precision == "fp64" else lcg.PREC_MIXED
    sp = lcg.SolveParams(1e-8, 2000, prec, 1e-4 if prec == lcg.PREC_MIXED else 0.0, 30)
    prm = lcg.default_params(tol=1e-8, max_iter=2000, precision=prec, inner_tol=1e-4)
    for A_case, gop, bb in ((oracle.from_stencil(op), good_op, b_nan), (oracle.from_stencil(bad), bad_op, b)):
        _, st_o, _, _ = oracle.pcg(A_case, bb, np.zeros(op.n), tol=1e-8, maxit=2000)
        assert st_o == oracle.BREAKDOWN
        _, sr, _ = oracle.solve_local_then_global(A_case, bb, np.zeros(op.n), tol=1e-8, maxit=2000)
        assert sr["status"] == oracle.BREAKDOWN
        # (the status is read back when stats are asked for; without them the calls are asynchronous)
        for call in (lambda x, s: lcg.pcg_solve(ctx, gop, cu(bb), x, sp, s),
                     lambda x, s: lcg.solve_local_then_global(ctx, gop, cu(bb), x, prm, s)):
            s = lcg.Stats()
            with pytest.raises(lcg.LcError) as e:
                call(cu(np.zeros(op.n)), s)
            assert e.value.code == lcg.LC_ERR_BREAKDOWN and s.status == lcg.LC_ERR_BREAKDOWN
    # the context and a good operator still work
    A = oracle.from_stencil(op)
    for call in (lambda x, s: lcg.pcg_solve(ctx, good_op, cu(b), x, sp, s),
                 lambda x, s: lcg.solve_local_then_global(ctx, good_op, cu(b), x, prm, s)):
        x = cu(np.zeros(op.n))
        s = lcg.Stats()
        call(x, s)
        assert s.status == 0 and oracle.relres(A, b, x.cpu().numpy()) <= 1e-8


@pytest.mark.parametrize("kind", ["stencil", "csr"])
def test_graph_replay_matches_direct_launches(kind):
    """Small systems run each solve call as a cached CUDA graph; the result
    and the statistics equal those of direct launches bit for bit, over
    repeated calls (replays) with changing data in the same buffers."""
    lcg.build()
    ctx = lcg.Context(0)
    cu = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)  # noqa: E731
    op = gen.random_stencil_2d(11, 50, 41)
    A = oracle.from_stencil(op)

    def make():
        if kind == "stencil":
            return lcg.StencilOperator(ctx, op.shape, cu(op.D), cu(op.Tx), cu(op.Ty))
        return lcg.CsrOperator(ctx, cu(A.rowptr, torch.int32), cu(A.col, torch.int32), cu(A.val))

    graphed, direct = make(), make()
    direct.set_tuning("graph_max_cells", 0)
    assert graphed.get_tuning("graph_max_cells") >= op.n
    rng = np.random.default_rng(3)
    prm = lcg.default_params(tol=1e-10)
    sp = lcg.SolveParams(1e-10, 100000, lcg.PREC_FP64, 0.0, 0)
    bg, bd, xg, xd = (cu(np.zeros(op.n)) for _ in range(4))
    for rep in range(3):
        x0 = 1.0 + 0.1 * rng.standard_normal(op.n)
        b = gen.csr_matvec(A.rowptr, A.col, A.val, x0)
        b[rng.integers(op.n)] += 1.0
        for call in ("alg1", "pcg"):
            res = []
            for gop, bb, xx in ((graphed, bg, xg), (direct, bd, xd)):
                bb.copy_(cu(b))
                xx.copy_(cu(x0))
                st = lcg.Stats()
                if call == "alg1":
                    lcg.solve_local_then_global(ctx, gop, bb, xx, prm, st)
                else:
                    lcg.pcg_solve(ctx, gop, bb, xx, sp, st)
                res.append((xx.cpu().numpy().copy(), st.as_dict()))
            (x1, s1), (x2, s2) = res
            assert np.array_equal(x1.view(np.int64), x2.view(np.int64)), (rep, call)
            for k in ("K", "nnzB", "it_local", "it_global", "restarts", "early_exit", "status"):
                assert s1[k] == s2[k], (rep, call, k)
            assert s1["relres_final"] == s2["relres_final"]
            assert oracle.relres(A, b, x1) <= 1e-10
