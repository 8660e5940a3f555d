"""Failure detection on the GPU without a fault: a grid barrier that cannot
complete (one arrival more than there are blocks) gives up after its short
limit, every block records LC_ERR_TIMEOUT and returns, the host reads the
status, and the context keeps working (a solve right after matches the
oracle)."""
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
