"""Gauss-Seidel smoothing of Alg 1 step 7 on the GPU against the oracle:
multicolour sweeps bit for bit (red-black on stencils, caller colourings on
CSR operators), and Alg 1 with smoothing within the solve tolerances."""
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


def csr_op(ctx, A):
    return lcg.CsrOperator(ctx, cu(A.rowptr, torch.int32), cu(A.col, torch.int32), cu(A.val))


SHAPES = [(7, 5, 1), (64, 16, 1), (65, 17, 1), (1, 40, 1), (40, 1, 1), (300, 260, 1), (5, 4, 3), (17, 9, 10),
          (33, 20, 7)]


def problem(k, shape):
    nx, ny, nz = shape
    op = gen.random_stencil_2d(k, nx, ny) if nz == 1 else gen.random_stencil_3d(k, nx, ny, nz)
    rng = np.random.default_rng(k + 70)
    return op, oracle.from_stencil(op), rng.standard_normal(op.n), rng.standard_normal(op.n)


def greedy_colouring(A):
    """Smallest colour not taken by an earlier neighbour (a proper colouring)."""
    col = np.zeros(A.n, np.uint8)
    for i in range(A.n):
        taken = {int(col[j]) for j in A.col[A.rowptr[i]:A.rowptr[i + 1]] if j < i}
        c = 0
        while c in taken:
            c += 1
        col[i] = c
    return col


@pytest.mark.parametrize("k,shape", list(enumerate(SHAPES)), ids=[f"{s[0]}x{s[1]}x{s[2]}" for s in SHAPES])
@pytest.mark.parametrize("sweeps", [1, 3])
def test_gs_stencil_bit_exact(ctx, k, shape, sweeps):
    op, A, b, x = problem(k, shape)
    col = gen.redblack_colouring(shape)
    ref = x
    for _ in range(sweeps):
        ref = oracle.gs_sweep(A, b, ref, col)
    xg = cu(x)
    lcg.gs_smooth(ctx, stencil_op(ctx, op), cu(b), xg, sweeps)
    assert np.array_equal(bits(xg.cpu().numpy()), bits(ref))


@pytest.mark.parametrize("k,shape", [(0, (64, 16, 1)), (1, (17, 9, 10)), (2, (65, 17, 1))])
@pytest.mark.parametrize("kind", ["redblack", "greedy"])
def test_gs_csr_bit_exact(ctx, k, shape, kind):
    op, A, b, x = problem(k, shape)
    col = gen.redblack_colouring(shape) if kind == "redblack" else greedy_colouring(A)
    ref = oracle.gs_sweep(A, b, oracle.gs_sweep(A, b, x, col), col)
    gop = csr_op(ctx, A)
    gop.set_colouring(cu(col, torch.uint8))
    xg = cu(x)
    lcg.gs_smooth(ctx, gop, cu(b), xg, 2)
    assert np.array_equal(bits(xg.cpu().numpy()), bits(ref))


def test_gs_rejects_bad_use(ctx):
    op, A, b, x = problem(3, (12, 10, 1))
    gop = csr_op(ctx, A)
    with pytest.raises(lcg.LcError) as e:
        lcg.gs_smooth(ctx, gop, cu(b), cu(x), 1)   # no colouring
    assert e.value.code == lcg.LC_ERR_UNSUPPORTED
    with pytest.raises(lcg.LcError):
        gop.set_colouring(cu(np.zeros(A.n), torch.uint8))   # neighbours share a colour
    with pytest.raises(lcg.LcError):
        gop.set_colouring(cu(gen.redblack_colouring((12, 10, 1)), torch.uint8), 1)   # colour out of range
    with pytest.raises(lcg.LcError):
        lcg.gs_smooth(ctx, stencil_op(ctx, op), cu(b), cu(x), 65)
    with pytest.raises(lcg.LcError):
        stencil_op(ctx, op).set_colouring(cu(gen.redblack_colouring((12, 10, 1)), torch.uint8))
    # zero sweeps leave x untouched
    xg = cu(x)
    lcg.gs_smooth(ctx, stencil_op(ctx, op), cu(b), xg, 0)
    assert np.array_equal(xg.cpu().numpy(), x)


@pytest.mark.parametrize("sweeps", [1, 2])
@pytest.mark.parametrize("operator", ["stencil", "csr"])
def test_local_then_global_with_gs_matches_oracle(ctx, sweeps, operator):
    d = gen.cfg1_heat2d(seed=11 + sweeps, n=96, radius=9)
    A = oracle.from_stencil(d["op"])
    col = gen.redblack_colouring(d["op"].shape)
    tol = 1e-8
    xr, sr, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], tol=tol, gs_sweeps=sweeps, colour=col)
    _, s0, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], tol=tol)
    assert sr["relres_tilde"] != s0["relres_tilde"]   # the smoothing acted
    if operator == "stencil":
        gop = stencil_op(ctx, d["op"])
    else:
        gop = csr_op(ctx, A)
        gop.set_colouring(cu(col, torch.uint8))
    prm = lcg.default_params(tol=tol, gs_sweeps=sweeps)
    x = cu(d["x0"])
    st = lcg.Stats()
    lcg.solve_local_then_global(ctx, gop, cu(d["b"]), x, prm, st)
    xg = x.cpu().numpy()
    assert st.K == sr["K"] and abs(st.it_local - sr["it_local"]) <= 1
    assert st.relres_tilde == pytest.approx(sr["relres_tilde"], rel=1e-6)
    assert abs(st.it_global - sr["it_global"]) <= 1
    assert oracle.relres(A, d["b"], xg) <= tol
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)
