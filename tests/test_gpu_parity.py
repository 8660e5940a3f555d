"""Parity of the CUDA path (through the C ABI) with the oracle.

Marking, expansion, thresholds and the extracted subsystem are compared bit
for bit; solves are compared within the tolerances the method states
(relative residual <= tol, solution within 1e-9 of the oracle's FP64 PCG run
with the same algorithm and tolerance).  Inputs are seeded (gen/); sizes
span several tiles of every kernel and ragged tails."""
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


def stencil_op(ctx, op: gen.Stencil):
    return lcg.StencilOperator(ctx, op.shape, cu(op.D), cu(op.Tx), cu(op.Ty), cu(op.Tz) if op.Tz is not None else None)


def csr_op(ctx, A: oracle.CSR):
    return lcg.CsrOperator(ctx, cu(A.rowptr, torch.int32), cu(A.col, torch.int32), cu(A.val))


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


SHAPES_2D = [(7, 5), (64, 16), (65, 17), (130, 37), (257, 9), (1, 40), (40, 1), (300, 260)]
SHAPES_3D = [(5, 4, 3), (16, 8, 8), (17, 9, 10), (33, 20, 7), (40, 1, 3)]


def problems():
    out = []
    for k, (nx, ny) in enumerate(SHAPES_2D):
        out.append((f"2d_{nx}x{ny}", gen.random_stencil_2d(k, nx, ny)))
    for k, (nx, ny, nz) in enumerate(SHAPES_3D):
        out.append((f"3d_{nx}x{ny}x{nz}", gen.random_stencil_3d(100 + k, nx, ny, nz)))
    return out


PROBLEMS = problems()


def rhs_and_x0(op, seed, local_source=True):
    rng = np.random.default_rng(seed)
    A = oracle.from_stencil(op)
    x_prev = 1.0 + 0.1 * rng.standard_normal(op.n)
    s = np.zeros(op.n)
    if local_source:
        idx = rng.choice(op.n, size=max(1, op.n // 50), replace=False)
        s[idx] = rng.uniform(0.5, 2.0, len(idx))
    b = gen.csr_matvec(A.rowptr, A.col, A.val, x_prev) + s + 1e-6 * rng.standard_normal(op.n)
    return A, b, x_prev


MARK_CASES = [
    (lcg.THR_REL_MAX, 1e-3, lcg.EXP_NONE, 0),
    (lcg.THR_REL_MAX, 1e-2, lcg.EXP_DILATE, 1),
    (lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2),
    (lcg.THR_REL_MAX, 0.2, lcg.EXP_DILATE, 7),
    (lcg.THR_EPS_NORMB, 1e-6, lcg.EXP_NONE, 0),
    (lcg.THR_EPS_NORMB, 1e-4, lcg.EXP_PAPER, 1),
    (lcg.THR_EPS_NORMB, 1e-5, lcg.EXP_PAPER, 6),
    (lcg.THR_REL_MAX, 0.05, lcg.EXP_PAPER, 3),
]


def run_mark(ctx, gop, b, x0, case):
    thr, prm, exp, rounds = case
    n = len(b)
    mask = torch.empty(n, dtype=torch.uint8, device=DEV)
    r0 = torch.empty(n, dtype=torch.float64, device=DEV)
    K = torch.zeros(1, dtype=torch.int32, device=DEV)
    tau = torch.zeros(1, dtype=torch.float64, device=DEV)
    lcg.mark_residual(ctx, gop, cu(b), cu(x0), lcg.MarkParams(thr, prm, exp, rounds), mask, K, r0, tau)
    torch.cuda.synchronize()
    return mask.cpu().numpy(), r0.cpu().numpy(), int(K.item()), float(tau.item())


@pytest.mark.parametrize("name,op", PROBLEMS, ids=[p[0] for p in PROBLEMS])
@pytest.mark.parametrize("case", MARK_CASES, ids=[f"thr{c[0]}_{c[1]}_exp{c[2]}x{c[3]}" for c in MARK_CASES])
def test_mark_residual_bit_exact(ctx, name, op, case):
    A, b, x0 = rhs_and_x0(op, 7)
    ref = oracle.mark_residual(A, b, x0, case[0], case[1], case[2], case[3])
    gop = stencil_op(ctx, op)
    mask, r0, K, tau = run_mark(ctx, gop, b, x0, case)
    assert np.array_equal(bits(r0), bits(ref["r"]))
    assert bits([tau])[0] == bits([ref["tau"]])[0]
    assert np.array_equal(mask, ref["mask"])
    assert K == ref["K"]
    # the same operator in CSR form gives the same bits
    cop = csr_op(ctx, A)
    mask2, r02, K2, tau2 = run_mark(ctx, cop, b, x0, case)
    assert np.array_equal(bits(r02), bits(ref["r"])) and np.array_equal(mask2, ref["mask"]) and K2 == K
    assert bits([tau2])[0] == bits([tau])[0]


def test_example1_on_gpu(ctx):
    e = gen.example1()
    A = oracle.csr(e["rowptr"], e["col"], e["val"])
    gop = csr_op(ctx, A)
    mask, r0, K, tau = run_mark(ctx, gop, e["b"], e["x0"], (lcg.THR_EPS_NORMB, 1e-5, lcg.EXP_PAPER, 6))
    ref = oracle.mark_residual(A, e["b"], e["x0"], oracle.THR_EPS_NORMB, 1e-5, oracle.EXP_PAPER, 6)
    assert list(np.flatnonzero(mask) + 1) == [1, 2, 3, 4, 5, 6] and K == 6
    assert bits([tau])[0] == bits([ref["tau"]])[0] and np.array_equal(bits(r0), bits(ref["r"]))


@pytest.mark.parametrize("name,op", PROBLEMS, ids=[p[0] for p in PROBLEMS])
@pytest.mark.parametrize("alpha,layers", [(0.0, 0), (0.3, 0), (0.05, 2), (1.0, 0), (0.5, 5)])
def test_mark_gradient_bit_exact(ctx, name, op, alpha, layers):
    A, b, x0 = rhs_and_x0(op, 3)
    x0 = x0.copy()
    x0[: max(1, op.n // 10)] = 1.0   # flat patch: g == 0 there
    ref = oracle.mark_gradient(A, x0, alpha, layers)
    for gop in (stencil_op(ctx, op), csr_op(ctx, A)):
        mask = torch.empty(op.n, dtype=torch.uint8, device=DEV)
        K = torch.zeros(1, dtype=torch.int32, device=DEV)
        gmax = torch.zeros(1, dtype=torch.float64, device=DEV)
        lcg.mark_gradient(ctx, gop, cu(x0), alpha, layers, mask, K, gmax)
        torch.cuda.synchronize()
        assert bits([gmax.item()])[0] == bits([ref["gmax"]])[0]
        assert np.array_equal(mask.cpu().numpy(), ref["mask"])
        assert int(K.item()) == ref["K"]


@pytest.mark.parametrize("name,op", PROBLEMS, ids=[p[0] for p in PROBLEMS])
@pytest.mark.parametrize("density", [0.0, 0.03, 0.3, 1.0])
def test_extract_bit_exact(ctx, name, op, density):
    A, b, x0 = rhs_and_x0(op, 11)
    rng = np.random.default_rng(int(density * 100))
    mask = (rng.uniform(size=op.n) < density).astype(np.uint8)
    ref = oracle.extract(A, mask, b, x0)
    for gop in (stencil_op(ctx, op), csr_op(ctx, A)):
        out = lcg.Subsystem.empty(gop)
        lcg.extract(ctx, gop, cu(mask, torch.uint8), cu(b), cu(x0), out)
        torch.cuda.synchronize()
        got = out.trimmed()
        assert got["K"] == ref["K"] and got["nnz"] == len(ref["B"].col)
        assert np.array_equal(got["g2l"], ref["g2l"]) and np.array_equal(got["l2g"], ref["l2g"])
        assert np.array_equal(got["rowptr"], ref["B"].rowptr) and np.array_equal(got["col"], ref["B"].col)
        assert np.array_equal(bits(got["val"]), bits(ref["B"].val))
        assert np.array_equal(bits(got["rhs"]), bits(ref["rhs"]))
        assert np.array_equal(bits(got["xL0"]), bits(ref["xL0"]))


SOLVE_PROBLEMS = [p for p in PROBLEMS if p[1].n >= 20]


@pytest.mark.parametrize("name,op", SOLVE_PROBLEMS, ids=[p[0] for p in SOLVE_PROBLEMS])
def test_pcg_matches_oracle(ctx, name, op):
    A, b, x0 = rhs_and_x0(op, 5)
    tol = 1e-8
    xr, st, it_ref, rr_ref = oracle.pcg(A, b, x0, tol=tol)
    assert st == oracle.OK
    for gop in (stencil_op(ctx, op), csr_op(ctx, A)):
        x = cu(x0)
        stats = lcg.Stats()
        lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(tol, 100000, lcg.PREC_FP64, 0.0, 0), stats)
        xg = x.cpu().numpy()
        assert oracle.relres(A, b, xg) <= tol
        assert abs(stats.it_global - it_ref) <= 1
        assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)
        assert stats.relres_final <= tol


SCALED_SHAPES = [(64, 16), (130, 37), (300, 260), (2, 50)]


@pytest.mark.parametrize("nx,ny", SCALED_SHAPES + [(128, 40), (4, 9)])
@pytest.mark.parametrize("scaled,wide,big,pairdot,lazy", [(0, 0, 1, 0, 0), (1, 0, 1, 0, 0), (1, 1, 1, 0, 0),
                                                           (0, 0, 0, 0, 0), (1, 1, 0, 0, 0), (1, 1, 1, 1, 0),
                                                           (1, 1, 0, 1, 0), (1, 1, 1, 1, 1), (1, 1, 0, 1, 1)])
def test_pcg_scaled_and_unscaled_match_oracle(ctx, nx, ny, scaled, wide, big, pairdot, lazy):
    """The 2-D FP64 solve on D^-1/2 A D^-1/2 (pcg_scaled = 1) and on A with the
    explicit Jacobi preconditioner (0) are the same Jacobi-PCG iteration in
    exact arithmetic: both match the oracle's iteration count within one and
    its solution within 1e-9, with 768-thread blocks (pcg_big) or 256, and
    with the dot products and block sums on FP32 pairs (pcg_pairdot) or in
    FP64, with x += alpha p carried by the next iteration's first phase
    (pcg_lazy_x) or not."""
    op = gen.random_stencil_2d(nx + 7 * ny, nx, ny)
    A, b, x0 = rhs_and_x0(op, 13)
    tol = 1e-9
    xr, st, it_ref, _ = oracle.pcg(A, b, x0, tol=tol)
    assert st == oracle.OK
    gop = stencil_op(ctx, op)
    gop.set_tuning("pcg_scaled", scaled)
    gop.set_tuning("pcg_wide", wide)
    gop.set_tuning("pcg_big", big)
    gop.set_tuning("pcg_pairdot", pairdot)
    gop.set_tuning("pcg_lazy_x", lazy)
    assert gop.get_tuning("pcg_scaled") == scaled and gop.get_tuning("pcg_wide") == wide
    assert gop.get_tuning("pcg_big") == big and gop.get_tuning("pcg_pairdot") == pairdot
    assert gop.get_tuning("pcg_lazy_x") == lazy
    x = cu(x0)
    stats = lcg.Stats()
    lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(tol, 100000, lcg.PREC_FP64, 0.0, 0), stats)
    xg = x.cpu().numpy()
    assert oracle.relres(A, b, xg) <= tol
    assert stats.relres_final <= tol
    assert abs(stats.it_global - it_ref) <= 1
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("pairdot,lazy", [(0, 0), (1, 0), (1, 1)])
def test_pcg_power_of_two_scale_invariance(ctx, dim, pairdot, lazy):
    """Scaling b and x0 by 2^k scales every FP64 quantity of the scaled 2-D
    and 3-D solves exactly, and the FP32 stopping norm and the FP32-pair dot products
    and block sums rescale with it (their exponent shifts follow b.b and
    r.z): the solution is 2^k times the unscaled one bit for bit, with the
    same iteration count, from 2^-400 to 2^400."""
    op = gen.random_stencil_2d(5, 64, 40) if dim == 2 else gen.random_stencil_3d(5, 24, 12, 10)
    A, b, x0 = rhs_and_x0(op, 29)
    gop = stencil_op(ctx, op)
    gop.set_tuning("pcg_pairdot", pairdot)
    gop.set_tuning("pcg_lazy_x", lazy)
    sp = lcg.SolveParams(1e-10, 100000, lcg.PREC_FP64, 0.0, 0)
    runs = {}
    for k in (0, -400, 400):
        x = cu(np.ldexp(x0, k))
        st = lcg.Stats()
        lcg.pcg_solve(ctx, gop, cu(np.ldexp(b, k)), x, sp, st)
        runs[k] = (x.cpu().numpy(), st.it_global)
    x_ref, it_ref = runs[0]
    assert oracle.relres(A, b, x_ref) <= 1e-10
    for k in (-400, 400):
        assert runs[k][1] == it_ref
        assert np.array_equal(bits(runs[k][0]), bits(np.ldexp(x_ref, k)))


@pytest.mark.parametrize("shape", [(16, 8, 8), (17, 9, 10), (33, 20, 7), (40, 1, 3), (5, 4, 3)])
@pytest.mark.parametrize("scaled,pairdot,lazy", [(0, 1, 1), (1, 0, 0), (1, 1, 0), (1, 1, 1)])
def test_pcg_3d_scaled_and_unscaled_match_oracle(ctx, shape, scaled, pairdot, lazy):
    """The 3D FP64 solve on D^-1/2 A D^-1/2 and on A with the explicit Jacobi
    preconditioner both match the oracle's Jacobi-PCG (iterations within one,
    solution within 1e-9); so does the 3D mixed-precision solve on the scaled
    system (relres 1e-10)."""
    op = gen.random_stencil_3d(sum(shape) + 3, *shape)
    A, b, x0 = rhs_and_x0(op, 17)
    tol = 1e-9
    xr, st, it_ref, _ = oracle.pcg(A, b, x0, tol=tol)
    gop = stencil_op(ctx, op)
    gop.set_tuning("pcg_scaled", scaled)
    gop.set_tuning("pcg_pairdot", pairdot)
    gop.set_tuning("pcg_lazy_x", lazy)
    x = cu(x0)
    stats = lcg.Stats()
    lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(tol, 100000, lcg.PREC_FP64, 0.0, 0), stats)
    xg = x.cpu().numpy()
    assert oracle.relres(A, b, xg) <= tol and abs(stats.it_global - it_ref) <= 1
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)
    x = cu(x0)
    lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(1e-10, 100000, lcg.PREC_MIXED, 1e-5, 30), stats)
    assert oracle.relres(A, b, x.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("shape", [(35, 11, 37), (9, 17, 33), (40, 17, 37), (64, 24, 20)])
@pytest.mark.parametrize("minblocks", [2, 3, 4])
def test_pcg_3d_several_z_tiles_and_register_budgets(ctx, shape, minblocks):
    """Grids deeper than one tile (16 planes) with a ragged last tile: the 3D
    march's plane-ahead pipeline crosses tile boundaries (p of the plane
    below and above a tile, the lazy x update only on the tile's own planes),
    at each register budget of the persistent kernel.  FP64 (default scaled
    kernel: iterations within one, solution within 1e-9 of the oracle) and
    mixed precision (relres 1e-10); with nx a multiple of 4 the FP32 inner
    solve streams its planes through shared memory by asynchronous copies
    across several blocks (halos that other blocks wrote)."""
    op = gen.random_stencil_3d(sum(shape) + minblocks, *shape)
    A, b, x0 = rhs_and_x0(op, 23)
    tol = 1e-9
    xr, st, it_ref, _ = oracle.pcg(A, b, x0, tol=tol)
    gop = stencil_op(ctx, op)
    gop.set_tuning("pcg_minblocks", minblocks)
    x = cu(x0)
    stats = lcg.Stats()
    lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(tol, 100000, lcg.PREC_FP64, 0.0, 0), stats)
    xg = x.cpu().numpy()
    assert oracle.relres(A, b, xg) <= tol and abs(stats.it_global - it_ref) <= 1
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)
    x = cu(x0)
    lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(1e-10, 100000, lcg.PREC_MIXED, 1e-5, 30), stats)
    assert oracle.relres(A, b, x.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("cscale,bscale", [(1e25, 1e35), (1e-25, 1e-30), (1.0, 1e-140), (1e5, 1e150),
                                            (1e45, 1e50), (1e-45, 1e-40)])
def test_pcg_scaled_extreme_magnitudes(ctx, cscale, bscale):
    """The scaled solve sums its stopping norm in FP32 with exponents shifted
    by ||b|| and max D, so coefficients and right-hand sides far outside
    FP32's range still stop at the FP64 tolerance (the oracle's iteration
    count within one)."""
    op0 = gen.random_stencil_2d(77, 96, 40)
    op = gen.Stencil(op0.shape, op0.D * cscale, op0.Tx * cscale, op0.Ty * cscale, None, op0.meta)
    A = oracle.from_stencil(op)
    rng = np.random.default_rng(3)
    b = rng.uniform(0.5, 1.5, op.n) * bscale
    x0 = np.zeros(op.n)
    tol = 1e-8
    xr, st, it_ref, _ = oracle.pcg(A, b, x0, tol=tol)
    assert st == oracle.OK
    gop = stencil_op(ctx, op)
    assert gop.get_tuning("pcg_scaled") == 1
    x = cu(x0)
    stats = lcg.Stats()
    lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(tol, 100000, lcg.PREC_FP64, 0.0, 0), stats)
    xg = x.cpu().numpy()
    assert oracle.relres(A, b, xg) <= tol
    assert abs(stats.it_global - it_ref) <= 1
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)


@pytest.mark.parametrize("nx,pairdot,lazy", [(33, 0, 0), (36, 0, 0), (36, 1, 0), (36, 1, 1)])
def test_pcg_edge_cases(ctx, nx, pairdot, lazy):
    op = gen.random_stencil_2d(1, nx, 21)
    A = oracle.from_stencil(op)
    gop = stencil_op(ctx, op)
    gop.set_tuning("pcg_pairdot", pairdot)
    gop.set_tuning("pcg_lazy_x", lazy)
    sp = lcg.SolveParams(1e-8, 100000, lcg.PREC_FP64, 0.0, 0)
    # b = 0 gives x = 0
    x = cu(np.ones(op.n))
    st = lcg.Stats()
    lcg.pcg_solve(ctx, gop, cu(np.zeros(op.n)), x, sp, st)
    assert not x.cpu().numpy().any() and st.it_global == 0
    # an exact start needs no iteration
    xs = np.random.default_rng(0).standard_normal(op.n)
    b = A.dense() @ xs
    xr, _, _, _ = oracle.pcg(A, b, np.zeros(op.n), tol=1e-14)
    x = cu(xr)
    lcg.pcg_solve(ctx, gop, cu(b), x, sp, st)
    assert st.it_global == 0 and st.early_exit == 1
    # max_iter reached: NOT_CONVERGED with stats filled
    x = cu(np.zeros(op.n))
    rc = lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(1e-14, 3, lcg.PREC_FP64, 0.0, 0), st,
                       allow_not_converged=True)
    assert rc == lcg.LC_ERR_NOT_CONVERGED and st.it_global == 3
    assert st.relres_final == pytest.approx(oracle.relres(A, b, x.cpu().numpy()), rel=1e-6)
    # ... and x is the third iterate (with pcg_lazy_x, the last update is flushed)
    x3, _, it3, _ = oracle.pcg(A, b, np.zeros(op.n), tol=1e-14, maxit=3)
    assert it3 == 3
    assert np.linalg.norm(x.cpu().numpy() - x3) <= 1e-12 * np.linalg.norm(x3)
    # a negative definite operator breaks down
    neg = oracle.csr(A.rowptr, A.col, -A.val)
    with pytest.raises(lcg.LcError):
        csr_op(ctx, neg)   # rejected at creation: non-positive diagonal


@pytest.mark.parametrize("mode", ["residual", "gradient", "paper"])
@pytest.mark.parametrize("n", [48, 128])
def test_local_then_global_matches_oracle(ctx, mode, n):
    d = gen.cfg1_heat2d(seed=n, n=n, radius=max(3, n // 12))
    A = oracle.from_stencil(d["op"])
    tol = 1e-8
    kw = dict(tol=tol)
    if mode == "residual":
        okw = dict(mark_mode=oracle.MARK_RESIDUAL, thr_mode=oracle.THR_REL_MAX, thr_param=1e-3,
                   exp_mode=oracle.EXP_DILATE, exp_rounds=2)
        prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2, tol=tol)
    elif mode == "paper":
        okw = dict(mark_mode=oracle.MARK_RESIDUAL, thr_mode=oracle.THR_EPS_NORMB, thr_param=1e-6,
                   exp_mode=oracle.EXP_PAPER, exp_rounds=2)
        prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_EPS_NORMB, 1e-6, lcg.EXP_PAPER, 2, tol=tol)
    else:
        okw = dict(mark_mode=oracle.MARK_GRADIENT, alpha=0.6, grad_layers=1)
        prm = lcg.default_params(lcg.MARK_GRADIENT, alpha=0.6, grad_layers=1, tol=tol)
    xr, sr, mask_r = oracle.solve_local_then_global(A, d["b"], d["x0"], **okw, **kw)
    for gop in (stencil_op(ctx, d["op"]), csr_op(ctx, A)):
        x = cu(d["x0"])
        st = lcg.Stats()
        lcg.solve_local_then_global(ctx, gop, cu(d["b"]), x, prm, st)
        xg = x.cpu().numpy()
        assert st.K == sr["K"] and st.nnzB == sr["nnzB"]
        assert abs(st.it_local - sr["it_local"]) <= 1
        assert st.early_exit == sr["early_exit"]
        assert oracle.relres(A, d["b"], xg) <= tol
        assert st.relres_tilde == pytest.approx(sr["relres_tilde"], rel=1e-6)
        assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)


@pytest.mark.parametrize("big,cap", [(1, 0), (0, 0), (1, 7), (0, 76), (1, 300)])
def test_local_grid_kernel_launch_shapes(ctx, big, cap):
    """The grid-wide local solve (cluster path off) with 768- or 256-thread
    blocks and 7 to 300 blocks: rows dealt to warps across all blocks, pair
    block sums; K, the local iteration count within one and the solution
    within 1e-9 of the oracle's Alg 1."""
    d = gen.cfg1_heat2d(seed=3, n=160, radius=30)
    A = oracle.from_stencil(d["op"])
    okw = dict(mark_mode=oracle.MARK_RESIDUAL, thr_mode=oracle.THR_REL_MAX, thr_param=1e-3,
               exp_mode=oracle.EXP_DILATE, exp_rounds=2)
    xr, sr, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], tol=1e-8, **okw)
    prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2, tol=1e-8)
    for gop in (stencil_op(ctx, d["op"]), csr_op(ctx, A)):
        gop.set_tuning("local_cluster_rows", 0)
        gop.set_tuning("pcg_big", big)
        gop.set_tuning("local_grid_cap", cap)
        assert gop.get_tuning("local_grid_cap") == cap
        x = cu(d["x0"])
        st = lcg.Stats()
        lcg.solve_local_then_global(ctx, gop, cu(d["b"]), x, prm, st)
        xg = x.cpu().numpy()
        assert st.K == sr["K"] > 0 and abs(st.it_local - sr["it_local"]) <= 1
        assert oracle.relres(A, d["b"], xg) <= 1e-8
        assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)


@pytest.mark.parametrize("n,radius,beta,rounds", [(96, 10, 1e-3, 2), (256, 40, 1e-3, 3), (384, 90, 1e-4, 4),
                                                   (300, 150, 1e-6, 8)])
@pytest.mark.parametrize("cluster,threads,single", [(1 << 30, 256, 0), (1 << 30, 1024, 0), (0, 256, 0), (0, 256, 1),
                                                    (0, 256, 2)])
def test_local_solve_cluster_and_grid_match_oracle(ctx, n, radius, beta, rounds, cluster, threads, single):
    """The local solve on one thread-block cluster (vectors in distributed
    shared memory), on the whole grid, on the whole grid with one reduction
    per iteration (single = 1) and pipelined with one barrier per iteration
    (single = 2) give the oracle's local iteration count within one and the
    same Alg 1 result; subsystems from a few hundred rows to more than the
    cluster holds (that one falls back to the grid kernel)."""
    d = gen.cfg1_heat2d(seed=n + radius, n=n, radius=radius)
    A = oracle.from_stencil(d["op"])
    tol = 1e-8
    xr, sr, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], thr_mode=oracle.THR_REL_MAX, thr_param=beta,
                                               exp_mode=oracle.EXP_DILATE, exp_rounds=rounds, tol=tol)
    prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, beta, lcg.EXP_DILATE, rounds, tol=tol)
    gop = stencil_op(ctx, d["op"])
    gop.set_tuning("local_cluster_rows", cluster)
    gop.set_tuning("local_cluster_threads", threads)
    gop.set_tuning("local_single", int(single == 1))
    gop.set_tuning("local_pipelined", int(single == 2))
    assert gop.get_tuning("local_cluster_rows") == cluster and gop.get_tuning("local_cluster_threads") == threads
    x = cu(d["x0"])
    st = lcg.Stats()
    lcg.solve_local_then_global(ctx, gop, cu(d["b"]), x, prm, st)
    xg = x.cpu().numpy()
    assert st.K == sr["K"] and st.nnzB == sr["nnzB"] and st.K > 0
    assert abs(st.it_local - sr["it_local"]) <= 1
    assert st.relres_tilde == pytest.approx(sr["relres_tilde"], rel=1e-6)
    assert oracle.relres(A, d["b"], xg) <= tol
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)


def test_local_solve_cluster_edge_sizes(ctx):
    """K = 0, 1, and a few rows (fewer rows than CTAs in the cluster): the
    cluster kernel's empty and ragged partitions."""
    op, A, b, x0, beta_for = edge_case_problem()
    gop = stencil_op(ctx, op)
    gop.set_tuning("local_cluster_rows", 1 << 30)
    for k in (1, 2, 5, 17):
        beta = beta_for(k)
        prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, beta, lcg.EXP_NONE, 0, tol=1e-9)
        xr, sr, _ = oracle.solve_local_then_global(A, b, x0, thr_mode=oracle.THR_REL_MAX, thr_param=beta,
                                                   exp_mode=oracle.EXP_NONE, exp_rounds=0, tol=1e-9)
        assert sr["K"] == k
        x = cu(x0)
        st = lcg.Stats()
        lcg.solve_local_then_global(ctx, gop, cu(b), x, prm, st)
        assert st.K == k and abs(st.it_local - sr["it_local"]) <= 1
        assert st.relres_tilde == pytest.approx(sr["relres_tilde"], rel=1e-6)
        assert oracle.relres(A, b, x.cpu().numpy()) <= 1e-9


def edge_case_problem():
    """A 64 x 48 operator and b = A x0 + s, s > 0 on 40 cells with distinct
    values, so the k largest residuals are separated by a threshold beta(k)."""
    op = gen.random_stencil_2d(5, 64, 48)
    A = oracle.from_stencil(op)
    rng = np.random.default_rng(8)
    x0 = 1.0 + 0.1 * rng.standard_normal(op.n)
    s = np.zeros(op.n)
    idx = rng.choice(op.n, size=40, replace=False)
    s[idx] = np.linspace(1.0, 2.0, 40)
    b = gen.csr_matvec(A.rowptr, A.col, A.val, x0) + s
    r = np.abs(b - gen.csr_matvec(A.rowptr, A.col, A.val, x0))
    order = np.argsort(-r, kind="stable")

    def beta_for(k):
        return float((r[order[k - 1]] + r[order[k]]) / 2 / r.max())

    return op, A, b, x0, beta_for


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pipelined_local_solve_edge_sizes(ctx, precision):
    """The pipelined grid kernel (cluster kernel off) on subsystems of 0, 1,
    2, 5 and 17 rows -- fewer rows than row warps, most threads without a row
    -- in FP64 and as the FP32 inner solve of mixed precision."""
    op, A, b, x0, beta_for = edge_case_problem()
    gop = stencil_op(ctx, op)
    gop.set_tuning("local_cluster_rows", 0)
    mixed = precision == "mixed"
    for k in (0, 1, 2, 5, 17):
        beta = 2.0 if k == 0 else beta_for(k)
        prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, beta, lcg.EXP_NONE, 0, tol=1e-9,
                                 precision=lcg.PREC_MIXED if mixed else lcg.PREC_FP64, inner_tol=1e-3)
        xr, sr, _ = oracle.solve_local_then_global(A, b, x0, thr_mode=oracle.THR_REL_MAX, thr_param=beta,
                                                   exp_mode=oracle.EXP_NONE, exp_rounds=0, tol=1e-9)
        assert sr["K"] == k
        x = cu(x0)
        st = lcg.Stats()
        lcg.solve_local_then_global(ctx, gop, cu(b), x, prm, st)
        assert st.K == k and st.status == 0
        if not mixed:
            assert abs(st.it_local - sr["it_local"]) <= 1
            assert st.relres_tilde == pytest.approx(sr["relres_tilde"], rel=1e-6)
        assert oracle.relres(A, b, x.cpu().numpy()) <= 1e-9


def test_local_then_global_edge_K_zero_and_full(ctx):
    d = gen.cfg1_heat2d(seed=2, n=40, radius=4)
    A = oracle.from_stencil(d["op"])
    gop = stencil_op(ctx, d["op"])
    for beta, rounds in [(2.0, 0), (0.0, 60)]:
        prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, beta, lcg.EXP_DILATE, rounds, tol=1e-9)
        xr, sr, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], thr_param=beta, exp_rounds=rounds, tol=1e-9)
        x = cu(d["x0"])
        st = lcg.Stats()
        lcg.solve_local_then_global(ctx, gop, cu(d["b"]), x, prm, st)
        assert st.K == sr["K"] and st.early_exit == sr["early_exit"]
        assert oracle.relres(A, d["b"], x.cpu().numpy()) <= 1e-9


def test_nan_handling_matches_oracle(ctx):
    op = gen.random_stencil_2d(4, 70, 33)
    A, b, x0 = rhs_and_x0(op, 9)
    b = b.copy()
    b[5] = np.nan
    x0 = x0.copy()
    x0[1000] = np.nan
    for case in [(lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2), (lcg.THR_REL_MAX, 1e-2, lcg.EXP_PAPER, 2)]:
        ref = oracle.mark_residual(A, b, x0, *case)
        mask, r0, K, tau = run_mark(ctx, stencil_op(ctx, op), b, x0, case)
        assert np.array_equal(mask, ref["mask"]) and K == ref["K"]
        assert bits([tau])[0] == bits([ref["tau"]])[0]
    ref = oracle.mark_gradient(A, x0, 0.1, 1)
    mask = torch.empty(op.n, dtype=torch.uint8, device=DEV)
    K = torch.zeros(1, dtype=torch.int32, device=DEV)
    lcg.mark_gradient(ctx, stencil_op(ctx, op), cu(x0), 0.1, 1, mask, K)
    assert np.array_equal(mask.cpu().numpy(), ref["mask"])


# ---------------------------------------------------------------- mixed precision (FP32 inner, FP64 refinement)

MIXED = [p for p in PROBLEMS if p[1].n >= 20]


@pytest.mark.parametrize("name,op", MIXED, ids=[p[0] for p in MIXED])
def test_mixed_precision_pcg_reaches_fp64_tolerance(ctx, name, op):
    """FP32 inner CG inside FP64 refinement reaches the FP64 relative residual
    of the plain FP64 solve; its error against the oracle's FP64 solution is
    stated (and bounded loosely by the conditioning).  Stencil operators with
    768- and 256-thread blocks (pcg_big 1 and 0), and CSR."""
    A, b, x0 = rhs_and_x0(op, 21)
    tol = 1e-10
    xr, st, _, _ = oracle.pcg(A, b, x0, tol=1e-13)
    small = stencil_op(ctx, op)
    small.set_tuning("pcg_big", 0)
    for gop in (stencil_op(ctx, op), small, csr_op(ctx, A)):
        x = cu(x0)
        stats = lcg.Stats()
        lcg.pcg_solve(ctx, gop, cu(b), x, lcg.SolveParams(tol, 100000, lcg.PREC_MIXED, 1e-4, 30), stats)
        xg = x.cpu().numpy()
        rr = oracle.relres(A, b, xg)
        assert rr <= tol, rr
        assert stats.restarts >= 1 and stats.relres_final <= tol
        err = np.linalg.norm(xg - xr) / np.linalg.norm(xr)
        assert err <= 1e-7, err


def test_mixed_precision_local_then_global(ctx):
    d = gen.cfg1_heat2d(seed=9, n=96, radius=8)
    A = oracle.from_stencil(d["op"])
    xr, sr, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], tol=1e-8)
    for gop in (stencil_op(ctx, d["op"]), csr_op(ctx, A)):
        x = cu(d["x0"])
        st = lcg.Stats()
        lcg.solve_local_then_global(ctx, gop, cu(d["b"]), x, lcg.default_params(tol=1e-8, precision=lcg.PREC_MIXED,
                                                                                 inner_tol=1e-4), st)
        xg = x.cpu().numpy()
        assert st.K == sr["K"]
        assert oracle.relres(A, d["b"], xg) <= 1e-8
        assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr)


def test_mixed_precision_rejects_bad_parameters(ctx):
    op = gen.random_stencil_2d(1, 16, 16)
    gop = stencil_op(ctx, op)
    x = cu(np.zeros(op.n))
    for bad in [lcg.SolveParams(1e-8, 100, lcg.PREC_MIXED, 0.0, 10), lcg.SolveParams(1e-8, 100, lcg.PREC_MIXED, 1e-4, 0),
                lcg.SolveParams(1e-8, 100, 7, 1e-4, 10)]:
        with pytest.raises(lcg.LcError) as e:
            lcg.pcg_solve(ctx, gop, cu(np.ones(op.n)), x, bad)
        assert e.value.code == lcg.LC_ERR_INVALID_ARG


@pytest.mark.parametrize("cap", [0, 5, 13])
def test_pipelined_local_solve_row_state_in_shared_and_global_memory(ctx, cap):
    """The pipelined local solve keeps a thread's rows in shared memory when
    every thread has at most three rows, else in global memory; a capped grid
    (5 or 13 blocks of 15 row warps: 2,400 or 6,240 rows per row round)
    sends the same 49,365-row subsystem down the global-memory path, with
    ragged last rounds.  Both against the oracle's Alg 1."""
    d = gen.cfg1_heat2d(seed=440, n=320, radius=120)
    A = oracle.from_stencil(d["op"])
    tol = 1e-8
    okw = dict(thr_mode=oracle.THR_REL_MAX, thr_param=1e-6, exp_mode=oracle.EXP_DILATE, exp_rounds=6)
    xr, sr, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], tol=tol, **okw)
    prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-6, lcg.EXP_DILATE, 6, tol=tol)
    gop = stencil_op(ctx, d["op"])
    gop.set_tuning("local_cluster_rows", 0)
    gop.set_tuning("local_grid_cap", cap)
    x = cu(d["x0"])
    st = lcg.Stats()
    lcg.solve_local_then_global(ctx, gop, cu(d["b"]), x, prm, st)
    xg = x.cpu().numpy()
    assert st.K == sr["K"] and (cap == 0 or st.K > 3 * 32 * 15 * cap)
    assert abs(st.it_local - sr["it_local"]) <= 1 and abs(st.it_global - sr["it_global"]) <= 1
    assert oracle.relres(A, d["b"], xg) <= tol
    assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)


@pytest.mark.parametrize("mode", ["residual", "gradient"])
@pytest.mark.parametrize("single", [0, 1, 2])
def test_local_single_reduction_on_csr_and_stencil(ctx, mode, single):
    """Alg 1 with the single-reduction local solve (single = 1) and the
    pipelined one (single = 2; one grid barrier per CG iteration) against the
    oracle, on stencil and CSR operators."""
    d = gen.cfg1_heat2d(seed=21, n=160, radius=14)
    A = oracle.from_stencil(d["op"])
    tol = 1e-8
    if mode == "residual":
        okw = dict(mark_mode=oracle.MARK_RESIDUAL, thr_mode=oracle.THR_REL_MAX, thr_param=1e-3,
                   exp_mode=oracle.EXP_DILATE, exp_rounds=2)
        prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2, tol=tol)
    else:
        okw = dict(mark_mode=oracle.MARK_GRADIENT, alpha=0.3, grad_layers=2)
        prm = lcg.default_params(lcg.MARK_GRADIENT, alpha=0.3, grad_layers=2, tol=tol)
    xr, sr, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], tol=tol, **okw)
    for gop in (stencil_op(ctx, d["op"]), csr_op(ctx, A)):
        gop.set_tuning("local_single", int(single == 1))
        gop.set_tuning("local_pipelined", int(single == 2))
        gop.set_tuning("local_cluster_rows", 0)
        x = cu(d["x0"])
        st = lcg.Stats()
        lcg.solve_local_then_global(ctx, gop, cu(d["b"]), x, prm, st)
        xg = x.cpu().numpy()
        assert st.K == sr["K"] and abs(st.it_local - sr["it_local"]) <= 1
        assert abs(st.it_global - sr["it_global"]) <= 1
        assert st.relres_tilde == pytest.approx(sr["relres_tilde"], rel=1e-6)
        assert oracle.relres(A, d["b"], xg) <= tol
        assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)
