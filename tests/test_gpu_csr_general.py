"""General CSR operators through the CSR path: 9-point diffusion (the pattern
of the paper's deforming-mesh systems) and 3T-like coupled systems (three
interleaved temperatures per cell, 3 x 3 block coupling).  Marking,
expansion and the extracted subsystem bit for bit against the oracle;
Jacobi-PCG, Alg 1 and mixed precision within the solve tolerances;
multicolour Gauss-Seidel with a greedy colouring bit for bit."""
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


CASES = [("ninepoint", 64, 48), ("ninepoint", 130, 37), ("ninepoint", 1, 50), ("threeT", 40, 30), ("threeT", 97, 61),
         ("threeT", 5, 1)]


def problem(kind, nx, ny, seed=0):
    rp, ci, av = (gen.ninepoint_2d if kind == "ninepoint" else gen.threeT_2d)(seed + nx * 3 + ny, nx, ny)
    A = oracle.csr(rp, ci, av)
    rng = np.random.default_rng(nx + 7 * ny + seed)
    x0 = 1.0 + 0.1 * rng.standard_normal(A.n)
    s = np.zeros(A.n)
    idx = rng.choice(A.n, size=max(1, A.n // 60), replace=False)
    s[idx] = rng.uniform(0.5, 2.0, len(idx))
    b = gen.csr_matvec(rp, ci, av, x0) + s
    return A, b, x0


def csr_op(ctx, A):
    return lcg.CsrOperator(ctx, cu(A.rowptr, torch.int32), cu(A.col, torch.int32), cu(A.val))


IDS = [f"{k}_{nx}x{ny}" for k, nx, ny in CASES]


@pytest.mark.parametrize("kind,nx,ny", CASES, ids=IDS)
@pytest.mark.parametrize("case", [(lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2), (lcg.THR_EPS_NORMB, 1e-6, lcg.EXP_PAPER, 3)])
def test_marking_and_extraction_bit_exact(ctx, kind, nx, ny, case):
    A, b, x0 = problem(kind, nx, ny)
    gop = csr_op(ctx, A)
    ref = oracle.mark_residual(A, b, x0, *case)
    mask = torch.empty(A.n, dtype=torch.uint8, device=DEV)
    r0 = torch.empty(A.n, dtype=torch.float64, device=DEV)
    K = torch.zeros(1, dtype=torch.int32, device=DEV)
    tau = torch.zeros(1, dtype=torch.float64, device=DEV)
    lcg.mark_residual(ctx, gop, cu(b), cu(x0), lcg.MarkParams(*case), mask, K, r0, tau)
    torch.cuda.synchronize()
    m = mask.cpu().numpy()
    assert np.array_equal(m, ref["mask"]) and int(K.item()) == ref["K"]
    assert np.array_equal(bits(r0.cpu().numpy()), bits(ref["r"])) and bits([tau.item()])[0] == bits([ref["tau"]])[0]
    e = oracle.extract(A, m, b, x0)
    out = lcg.Subsystem.empty(gop)
    lcg.extract(ctx, gop, mask, cu(b), cu(x0), out)
    torch.cuda.synchronize()
    got = out.trimmed()
    assert got["K"] == e["K"] and np.array_equal(got["l2g"], e["l2g"]) and np.array_equal(got["g2l"], e["g2l"])
    assert np.array_equal(got["rowptr"], e["B"].rowptr) and np.array_equal(got["col"], e["B"].col)
    assert np.array_equal(bits(got["val"]), bits(e["B"].val)) and np.array_equal(bits(got["rhs"]), bits(e["rhs"]))
    assert np.array_equal(bits(got["xL0"]), bits(e["xL0"]))


@pytest.mark.parametrize("kind,nx,ny", CASES, ids=IDS)
def test_gradient_marking_bit_exact(ctx, kind, nx, ny):
    A, b, x0 = problem(kind, nx, ny)
    ref = oracle.mark_gradient(A, x0, 0.2, 1)
    mask = torch.empty(A.n, dtype=torch.uint8, device=DEV)
    K = torch.zeros(1, dtype=torch.int32, device=DEV)
    gmax = torch.zeros(1, dtype=torch.float64, device=DEV)
    lcg.mark_gradient(ctx, csr_op(ctx, A), cu(x0), 0.2, 1, mask, K, gmax)
    torch.cuda.synchronize()
    assert np.array_equal(mask.cpu().numpy(), ref["mask"]) and int(K.item()) == ref["K"]
    assert bits([gmax.item()])[0] == bits([ref["gmax"]])[0]


@pytest.mark.parametrize("kind,nx,ny", [c for c in CASES if c[1] * c[2] >= 20], ids=[i for c, i in zip(CASES, IDS)
                                                                                     if c[1] * c[2] >= 20])
def test_pcg_and_alg1_match_oracle(ctx, kind, nx, ny):
    A, b, x0 = problem(kind, nx, ny)
    gop = csr_op(ctx, A)
    tol = 1e-8
    xr, st_r, it_r, _ = oracle.pcg(A, b, x0, tol=tol)
    x = cu(x0)
    st = lcg.Stats()
    lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(tol, 100000, lcg.PREC_FP64, 0.0, 0), st)
    xg = x.cpu().numpy()
    assert abs(st.it_global - it_r) <= 1 and oracle.relres(A, b, xg) <= tol
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)
    xa, sa, _ = oracle.solve_local_then_global(A, b, x0, tol=tol)
    x = cu(x0)
    lcg.solve_local_then_global(ctx, gop, cu(b), x, lcg.default_params(tol=tol), st)
    xg = x.cpu().numpy()
    assert st.K == sa["K"] and st.nnzB == sa["nnzB"] and abs(st.it_local - sa["it_local"]) <= 1
    assert abs(st.it_global - sa["it_global"]) <= 1 and oracle.relres(A, b, xg) <= tol
    assert np.linalg.norm(xg - xa) <= 1e-9 * np.linalg.norm(xa)
    # mixed precision reaches the FP64 tolerance too
    x = cu(x0)
    lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(1e-10, 100000, lcg.PREC_MIXED, 1e-4, 30), st)
    assert oracle.relres(A, b, x.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("kind,nx,ny", [("threeT", 97, 61), ("ninepoint", 130, 37)])
def test_csr_store_p_is_bit_identical(ctx, kind, nx, ny):
    """The global CSR solve with p stored once per row (csr_store_p 1, the
    default) and with p recomputed at every column (0) performs the same
    operations on the same values: identical iterations and bits of x, FP64
    and mixed precision; both match the oracle."""
    A, b, x0 = problem(kind, nx, ny)
    gop = csr_op(ctx, A)
    xr, _, it_r, _ = oracle.pcg(A, b, x0, tol=1e-8)
    out = {}
    for sp in (1, 0):
        gop.set_tuning("csr_store_p", sp)
        res = []
        for prm in (lcg.SolveParams(1e-8, 100000, lcg.PREC_FP64, 0.0, 0),
                    lcg.SolveParams(1e-10, 100000, lcg.PREC_MIXED, 1e-4, 30)):
            x = cu(x0)
            st = lcg.Stats()
            lcg.pcg_solve(ctx, gop, cu(b), x, prm, st)
            res.append((x.cpu().numpy(), st.it_global))
        out[sp] = res
    for k in range(2):
        assert out[0][k][1] == out[1][k][1]
        assert np.array_equal(bits(out[0][k][0]), bits(out[1][k][0]))
    assert abs(out[1][0][1] - it_r) <= 1
    assert np.linalg.norm(out[1][0][0] - xr) <= 1e-9 * np.linalg.norm(xr)


@pytest.mark.parametrize("kind,nx,ny", CASES, ids=IDS)
def test_gs_greedy_colouring_bit_exact(ctx, kind, nx, ny):
    A, b, x0 = problem(kind, nx, ny)
    col = gen.greedy_colouring(A.rowptr, A.col)
    ref = oracle.gs_sweep(A, b, oracle.gs_sweep(A, b, x0, col), col)
    gop = csr_op(ctx, A)
    gop.set_colouring(cu(col, torch.uint8))
    x = cu(x0)
    lcg.gs_smooth(ctx, gop, cu(b), x, 2)
    assert np.array_equal(bits(x.cpu().numpy()), bits(ref))
