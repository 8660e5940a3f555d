"""Multi-group stand-in (the structure of the paper's multi-group radiation
diffusion systems, Sec. 3.3, on synthetic data): 64 group systems on one
88 x 80 mesh with a shared sparsity pattern, solved together by the batched
Alg 1 (one launch) and compared group by group with the oracle: the local
domain and the subsystem equal the oracle's bit for bit, each group reaches relres
1e-8 (evaluated by the oracle), and its distance to the oracle's FP64
solution is bounded."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2001_01158_gb300 as lcg

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def groups():
    lcg.build()
    ctx = lcg.Context(0)
    items = gen.mg_standin(seed=3)
    systems = [(d["op"].shape[0], d["op"].shape[1], cu(d["op"].D), cu(d["op"].Tx), cu(d["op"].Ty)) for d in items]
    batch = lcg.Batch(ctx, systems)
    return ctx, items, batch, cu(np.concatenate([d["b"] for d in items])), cu(np.concatenate([d["x0"] for d in items]))


@pytest.mark.parametrize("cluster", [1, 4])
def test_multigroup_batched_matches_oracle(groups, cluster):
    """One CTA per group, and clusters of 4 CTAs per group."""
    ctx, items, batch, b, x0 = groups
    tol = 1e-8
    batch.set_tuning("cluster", cluster)
    batch.set_tuning("big_cells", 4096)
    x = x0.clone()
    batch.solve(b, x, lcg.batch_params(beta=1e-3, layers=2, tol=tol, inner_tol=1e-4))
    st = batch.stats()
    xs = x.cpu().numpy()
    for g, d in enumerate(items):
        A = oracle.from_stencil(d["op"])
        xr, sr, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], thr_mode=oracle.THR_REL_MAX, thr_param=1e-3,
                                                   exp_mode=oracle.EXP_DILATE, exp_rounds=2, tol=tol)
        assert st[g]["K"] == sr["K"] > 0 and st[g]["nnzB"] == sr["nnzB"], g
        assert st[g]["tau"] == sr["tau"], g
        m = oracle.mark_residual(A, d["b"], d["x0"], oracle.THR_REL_MAX, 1e-3, oracle.EXP_DILATE, 2)
        ex = oracle.extract(A, m["mask"], d["b"], d["x0"])
        dom = batch.domain(g)
        assert np.array_equal(dom["mask"], m["mask"]) and np.array_equal(dom["g2l"], ex["g2l"]), g
        assert np.array_equal(dom["col"], ex["B"].col) and np.array_equal(dom["rowptr"], ex["B"].rowptr), g
        assert np.array_equal(dom["val"].view(np.int64), ex["B"].val.view(np.int64)), g
        assert np.array_equal(dom["rhs"].view(np.int64), ex["rhs"].view(np.int64)), g
        xg = xs[batch.offsets[g]:batch.offsets[g + 1]]
        assert oracle.relres(A, d["b"], xg) <= tol, g
        assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr), g


def test_multigroup_sequential_fp64_alg1_matches_oracle(groups):
    """The same groups one after another through the FP64 Alg 1 entry point."""
    ctx, items, batch, b, x0 = groups
    for g in (0, 31, 63):
        d = items[g]
        A = oracle.from_stencil(d["op"])
        xr, sr, _ = oracle.solve_local_then_global(A, d["b"], d["x0"], tol=1e-8)
        gop = lcg.StencilOperator(ctx, d["op"].shape, cu(d["op"].D), cu(d["op"].Tx), cu(d["op"].Ty))
        x = cu(d["x0"])
        st = lcg.Stats()
        lcg.solve_local_then_global(ctx, gop, cu(d["b"]), x, lcg.default_params(tol=1e-8), st)
        xg = x.cpu().numpy()
        assert st.K == sr["K"] and abs(st.it_local - sr["it_local"]) <= 1 and abs(st.it_global - sr["it_global"]) <= 1
        assert np.linalg.norm(xg - xr) <= 1e-9 * np.linalg.norm(xr)
