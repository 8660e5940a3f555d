"""The nonlinear 2D heat problem of Sec. 3.2 on the GPU against the oracle:
the Picard-linearised system bit for bit from given conductivities, and
Picard-iterated time steps by the global PCG and by Alg 1 (both markings)
within the solve tolerances."""
import numpy as np
import pytest
import torch

import oracle
import paper_2001_01158_gb300 as lcg

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
DIR, NEU = lcg.BC_DIRICHLET, lcg.BC_NEUMANN


@pytest.fixture(scope="module")
def ctx():
    lcg.build()
    return lcg.Context(0)


def cu(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def e1_initial(n):
    """T0 = exp(-100 x) T_l + T_r at the cell centres of n x n cells on the unit square."""
    xc = (np.arange(n) + 0.5) / n
    return np.tile(np.exp(-100.0 * xc) * 1.0 + 1e-4, n)


BCS = [([DIR, DIR, NEU, NEU], [1.0, 1e-4, 0.0, 0.0]), ([NEU] * 4, [0.0] * 4), ([DIR] * 4, [0.3, 2.0, -1.0, 0.5]),
       ([NEU, DIR, DIR, NEU], [0.0, 1.5, 0.25, 0.0])]


@pytest.mark.parametrize("shape", [(99, 99), (64, 33), (1, 7), (7, 1)])
@pytest.mark.parametrize("bc", range(len(BCS)))
def test_heat_assemble_bit_exact(ctx, shape, bc):
    nx, ny = shape
    rng = np.random.default_rng(nx * 7 + ny + bc)
    kappa = 10 ** rng.uniform(-4, 1, nx * ny)
    Tn = rng.uniform(0, 1, nx * ny)
    h, dt = 1.0 / nx, 1e-2
    bt, bv = BCS[bc]
    A, b_ref = oracle.heat2d_system(nx, ny, h, dt, bt, bv, kappa, Tn)
    D, Tx, Ty, b = (torch.empty(nx * ny, dtype=torch.float64, device=DEV) for _ in range(4))
    lcg.heat2d_assemble(ctx, shape, h, dt, bt, bv, cu(kappa), cu(Tn), D, Tx, Ty, b)
    torch.cuda.synchronize()
    # the stencil arrays as CSR entries of the oracle's matrix
    M = A.dense()
    idx = np.arange(nx * ny)
    assert np.array_equal(bits(D.cpu().numpy()), bits(M[idx, idx]))
    east = idx[(idx % nx) + 1 < nx]
    north = idx[idx // nx + 1 < ny]
    Txh, Tyh = Tx.cpu().numpy(), Ty.cpu().numpy()
    assert np.array_equal(bits(Txh[east]), bits(-M[east, east + 1]))
    assert np.array_equal(bits(Tyh[north]), bits(-M[north, north + nx]))
    assert not Txh[np.setdiff1d(idx, east)].any() and not Tyh[np.setdiff1d(idx, north)].any()
    assert np.array_equal(bits(b.cpu().numpy()), bits(b_ref))


def heat_setup(ctx, n, T0, p=3.5):
    bt, bv = BCS[0]
    h, dt = 1.0 / n, 1e-2
    D, Tx, Ty, b = (torch.empty(n * n, dtype=torch.float64, device=DEV) for _ in range(4))
    lcg.heat2d_assemble(ctx, (n, n), h, dt, bt, bv, cu(T0 ** p), cu(T0), D, Tx, Ty, b)
    op = lcg.StencilOperator(ctx, (n, n, 1), D, Tx, Ty)
    return op, D, Tx, Ty, b, torch.empty(2 * n * n, dtype=torch.float64, device=DEV)


METHODS = {
    "global": dict(method=0),
    "residual": dict(method=1, mark_mode=oracle.MARK_RESIDUAL, thr_mode=oracle.THR_EPS_NORMB, thr_param=1e-10,
                     exp_mode=oracle.EXP_PAPER, exp_rounds=1),
    "gradient": dict(method=1, mark_mode=oracle.MARK_GRADIENT, alpha=1e-4, grad_layers=0),
    "residual_gs1": dict(method=1, mark_mode=oracle.MARK_RESIDUAL, thr_mode=oracle.THR_EPS_NORMB, thr_param=1e-10,
                         exp_mode=oracle.EXP_PAPER, exp_rounds=1, gs_sweeps=1),
}


def gpu_params(m):
    kw = METHODS[m]
    if kw.get("mark_mode", 0) == oracle.MARK_GRADIENT:
        prm = lcg.default_params(lcg.MARK_GRADIENT, alpha=kw["alpha"], grad_layers=kw["grad_layers"], tol=1e-10)
    else:
        prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_EPS_NORMB, 1e-10, lcg.EXP_PAPER, 1, tol=1e-10,
                                 gs_sweeps=kw.get("gs_sweeps", 0))
    return lcg.heat_params(1.0 / 99, 1e-2, 3.5, BCS[0][0], BCS[0][1], method=kw["method"], params=prm)


@pytest.mark.parametrize("method", list(METHODS))
def test_heat_steps_match_oracle(ctx, method):
    """Three time steps of the paper's 99 x 99 problem: every step's T within
    1e-8 of the oracle's (the paper's methods differ by <= 7.6e-9), Picard
    counts within one."""
    n = 99
    T0 = e1_initial(n)
    op, D, Tx, Ty, b, work = heat_setup(ctx, n, T0)
    hp = gpu_params(method)
    Tg = cu(T0)
    Tr = T0.copy()
    for step in range(3):
        Tn_g = Tg.clone()
        st = lcg.heat2d_step(ctx, op, hp, Tn_g, Tg, D, Tx, Ty, b, work)
        Tr, sr = oracle.heat2d_step(n, n, 1.0 / n, 1e-2, 3.5, BCS[0][0], BCS[0][1], Tr.copy(), **METHODS[method])
        T = Tg.cpu().numpy()
        assert st.status == 0 and sr["status"] == oracle.OK
        assert abs(st.picard_its - sr["picard_its"]) <= 1
        assert np.linalg.norm(T - Tr) / np.linalg.norm(Tr) <= 1e-8
        if METHODS[method]["method"] == 1:
            assert st.K_sum > 0


def test_heat_step_rejects_bad_use(ctx):
    n = 16
    T0 = e1_initial(n)
    op, D, Tx, Ty, b, work = heat_setup(ctx, n, T0)
    hp = gpu_params("global")
    T = cu(T0)
    other = torch.empty_like(D)
    with pytest.raises(lcg.LcError):
        lcg.heat2d_step(ctx, op, hp, cu(T0), T, other, Tx, Ty, b, work)   # not the operator's arrays
    bad = gpu_params("global")
    bad.bc_type[1] = 7
    with pytest.raises(lcg.LcError):
        lcg.heat2d_step(ctx, op, bad, cu(T0), T, D, Tx, Ty, b, work)
    bad = gpu_params("global")
    bad.max_picard = 0
    with pytest.raises(lcg.LcError):
        lcg.heat2d_step(ctx, op, bad, cu(T0), T, D, Tx, Ty, b, work)
    with pytest.raises(lcg.LcError):
        lcg.heat2d_assemble(ctx, (n, n), 0.0, 1e-2, BCS[0][0], BCS[0][1], cu(T0), cu(T0), D, Tx, Ty, b)
