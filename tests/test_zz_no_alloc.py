"""The allocation-free marking entry point agrees with lc_mark_residual.

Callers that cannot allocate device memory (inside another framework's pool,
under a fixed budget, or after start-up) use
lc_mark_residual_stencil_noalloc, whose scratch is a fixed device array in
the library.  This test calls it through the C ABI twice in a row on every case
-- so the second call runs on the scratch the first one left behind, and
each case after the first on what a case of another size and mode left --
and checks that each result equals, bit for bit, the result of
lc_mark_residual on an operator created the usual way.  It lives in its own file, collected last,
and builds everything it needs itself."""
import numpy as np
import pytest
import torch

import gen
import paper_2001_01158_gb300 as lcg

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


def _inputs(op, seed):
    # b = A x0 + a sparse source: the residual of x0 is local
    rng = np.random.default_rng(seed)
    x0 = 1.0 + 0.1 * rng.standard_normal(op.n)
    rp, ci, av = gen.stencil_to_csr(op)
    b = gen.csr_matvec(rp, ci, av, x0) + rng.standard_normal(op.n) * (rng.uniform(size=op.n) < 0.02)
    return b, x0


def _with_operator(ctx, op, b, x0, params):
    gop = lcg.StencilOperator(ctx, op.shape, _t(op.D), _t(op.Tx), _t(op.Ty), _t(op.Tz) if op.Tz is not None else None)
    mask = torch.empty(op.n, dtype=torch.uint8, device=DEV)
    r0 = torch.empty(op.n, dtype=torch.float64, device=DEV)
    K = torch.zeros(1, dtype=torch.int32, device=DEV)
    tau = torch.zeros(1, dtype=torch.float64, device=DEV)
    lcg.mark_residual(ctx, gop, _t(b), _t(x0), params, mask, K, r0, tau)
    torch.cuda.synchronize()
    return mask.cpu().numpy(), r0.cpu().numpy(), int(K.item()), float(tau.item())


def _without_allocation(op, b, x0, params):
    mask = torch.full((op.n,), 7, dtype=torch.uint8, device=DEV)
    r0 = torch.empty(op.n, dtype=torch.float64, device=DEV)
    K = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    tau = torch.zeros(1, dtype=torch.float64, device=DEV)
    lcg.mark_residual_stencil_noalloc(op.shape, _t(op.D), _t(op.Tx), _t(op.Ty),
                                      _t(op.Tz) if op.Tz is not None else None, _t(b), _t(x0), params, mask, r0, K,
                                      tau)
    torch.cuda.synchronize()
    return mask.cpu().numpy(), r0.cpu().numpy(), int(K.item()), float(tau.item())


def _same(a, b):
    m1, r1, k1, t1 = a
    m2, r2, k2, t2 = b
    assert np.array_equal(m1, m2)
    assert np.array_equal(r1.view(np.int64), r2.view(np.int64))
    assert k1 == k2
    assert np.float64(t1).view(np.int64) == np.float64(t2).view(np.int64)


def test_noalloc_matches_lc_mark_residual_on_two_calls_in_a_row():
    lcg.build()
    ctx = lcg.Context(0)
    cases = [
        (gen.random_stencil_2d(3, 300, 211), lcg.MarkParams(lcg.THR_EPS_NORMB, 1e-5, lcg.EXP_PAPER, 5)),
        (gen.random_stencil_2d(4, 129, 77), lcg.MarkParams(lcg.THR_REL_MAX, 1e-2, lcg.EXP_DILATE, 7)),
        (gen.random_stencil_3d(5, 33, 20, 9), lcg.MarkParams(lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 3)),
    ]
    for k, (op, params) in enumerate(cases):
        b, x0 = _inputs(op, k)
        ref = _with_operator(ctx, op, b, x0, params)
        assert 0 < ref[2] < op.n
        for _ in range(2):
            _same(_without_allocation(op, b, x0, params), ref)


def test_noalloc_rejects_grids_beyond_its_limit():
    lcg.build()
    n = lcg.LC_NOALLOC_MAX_CELLS + 1
    one = torch.zeros(1, dtype=torch.float64, device=DEV)
    with pytest.raises(lcg.LcError) as e:
        lcg.mark_residual_stencil_noalloc((n, 1, 1), one, one, one, None, one, one,
                                          lcg.MarkParams(lcg.THR_REL_MAX, 1e-3, lcg.EXP_NONE, 0),
                                          torch.zeros(1, dtype=torch.uint8, device=DEV), one,
                                          torch.zeros(1, dtype=torch.int32, device=DEV))
    assert e.value.code == lcg.LC_ERR_TOO_LARGE and "LC_NOALLOC_MAX_CELLS" in str(e.value)
