"""Batched Alg 1 (many uneven systems in one launch, CUDA graph, autotuner)
against the oracle, system by system: the local domain (mask) and the
extracted subsystem (g2l, l2g, B, rhs) equal the oracle's bit for bit, each
solution reaches the FP64 relative residual, and its error against the
oracle's FP64 solution is stated and bounded."""
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


def assert_domain_equal(batch, s, m, ex):
    """System s's mask and subsystem from the batched launch equal the
    oracle's marking m and extraction ex bit for bit."""
    g = batch.domain(s)
    assert np.array_equal(g["mask"], m["mask"]), s
    assert np.array_equal(g["g2l"], ex["g2l"]) and np.array_equal(g["l2g"], ex["l2g"]), s
    assert np.array_equal(g["rowptr"], ex["B"].rowptr) and np.array_equal(g["col"], ex["B"].col), s
    assert np.array_equal(g["val"].view(np.int64), ex["B"].val.view(np.int64)), s
    assert np.array_equal(g["rhs"].view(np.int64), ex["rhs"].view(np.int64)), s


def make_batch(seed, sides):
    rng = np.random.default_rng(seed)
    items = []
    for k, (nx, ny) in enumerate(sides):
        d = gen.cfg1_heat2d(seed=int(rng.integers(1 << 30)), n=max(nx, ny), radius=max(1.0, 0.15 * min(nx, ny)))
        if (nx, ny) != (d["op"].shape[0], d["op"].shape[1]):
            # rectangular system: random operator, local source
            op = gen.random_stencil_2d(int(rng.integers(1 << 30)), nx, ny)
            x0 = 1.0 + 0.1 * rng.standard_normal(op.n)
            src = np.zeros(op.n)
            src[rng.choice(op.n, size=max(1, op.n // 30), replace=False)] = 1.0
            d = {"op": op, "x0": x0, "b": gen.stencil_matvec(op, x0) + src}
        items.append(d)
    return items


SIDES = [(64, 64), (8, 8), (1, 50), (37, 1), (129, 70), (200, 200), (33, 17), (96, 96), (5, 300), (150, 149),
         (64, 65), (17, 33), (2, 2), (100, 3)]


@pytest.fixture(scope="module")
def setup():
    lcg.build()
    ctx = lcg.Context(0)
    items = make_batch(7, SIDES)
    systems = [(d["op"].shape[0], d["op"].shape[1], cu(d["op"].D), cu(d["op"].Tx), cu(d["op"].Ty)) for d in items]
    batch = lcg.Batch(ctx, systems)
    b = cu(np.concatenate([d["b"] for d in items]))
    x0 = cu(np.concatenate([d["x0"] for d in items]))
    return ctx, items, batch, b, x0


# (block, cluster, big_cells): one CTA per system, and thread-block clusters
# of 2, 4, 8 and 16 CTAs taking every system from big_cells cells on -- down to
# systems with fewer rows than the cluster has CTAs (empty row ranges)
CONFIGS = [(256, 1, 65536), (512, 1, 65536), (1024, 1, 65536), (1024, 2, 1000), (512, 4, 30), (1024, 8, 200),
           (1024, 16, 1)]


def set_config(batch, block, cluster, big):
    batch.set_tuning("block", block)
    batch.set_tuning("cluster", cluster)
    batch.set_tuning("big_cells", big)


@pytest.mark.parametrize("block,cluster,big", CONFIGS)
def test_batched_matches_oracle_per_system(setup, block, cluster, big):
    ctx, items, batch, b, x0 = setup
    tol = 1e-8
    prm = lcg.batch_params(beta=1e-3, layers=2, tol=tol, inner_tol=1e-4)
    set_config(batch, block, cluster, big)
    x = x0.clone()
    batch.solve(b, x, prm)
    st = batch.stats()
    xs = x.cpu().numpy()
    for s, d in enumerate(items):
        A = oracle.from_stencil(d["op"])
        m = oracle.mark_residual(A, d["b"], d["x0"], oracle.THR_REL_MAX, 1e-3, oracle.EXP_DILATE, 2)
        ex = oracle.extract(A, m["mask"], d["b"], d["x0"])
        assert st[s]["K"] == m["K"] and st[s]["nnzB"] == len(ex["B"].col), s
        assert st[s]["tau"] == m["tau"]
        assert_domain_equal(batch, s, m, ex)
        xg = xs[batch.offsets[s]:batch.offsets[s + 1]]
        assert oracle.relres(A, d["b"], xg) <= tol, s
        xr, _, _, _ = oracle.pcg(A, d["b"], d["x0"], tol=1e-13)
        assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr), s


@pytest.mark.parametrize("cluster", [1, 4])
def test_graph_replay_equals_direct_launch(setup, cluster):
    ctx, items, batch, b, x0 = setup
    prm = lcg.batch_params()
    set_config(batch, 512, cluster, 1000)
    x1 = x0.clone()
    batch.solve(b, x1, prm)
    torch.cuda.synchronize()
    x2 = x0.clone()
    batch.capture(b, x2, prm)
    for _ in range(2):   # replays start from whatever x holds: reset it each time
        x2.copy_(x0)
        batch.replay()
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)
    assert all(s["status"] == 0 for s in batch.stats())


def test_autotuner_picks_a_configuration(setup, tmp_path, monkeypatch):
    from paper_2001_01158_gb300 import autotune
    ctx, items, batch, b, x0 = setup
    monkeypatch.setenv("LC_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    cfg = autotune.tune_batch(batch, b, x0, lcg.batch_params())
    assert cfg["block"] in (256, 512, 1024) and len(cfg["candidates"]) == len(autotune.CANDIDATES)
    assert cfg["ms"] <= 1.03 * cfg["best_ms"]
    again = autotune.tune_batch(batch, b, x0, lcg.batch_params())   # from the cache
    assert all(again[k] == cfg[k] for k in autotune.KEYS)


def test_batched_rejects_unsupported_parameters(setup):
    ctx, items, batch, b, x0 = setup
    x = x0.clone()
    for p in [lcg.default_params(precision=lcg.PREC_FP64),
              lcg.default_params(lcg.MARK_GRADIENT, precision=lcg.PREC_MIXED),
              lcg.default_params(thr_mode=lcg.THR_EPS_NORMB, precision=lcg.PREC_MIXED)]:
        with pytest.raises(lcg.LcError) as e:
            batch.solve(b, x, p)
        assert e.value.code == lcg.LC_ERR_UNSUPPORTED


def test_batched_full_size_512_systems():
    """The bench's batched workload at its full size (512 systems, sides
    log-uniform in [64, 512], 35 M cells) in the launch configuration the
    bench times (autotuned, graph replay): every system reaches relres 1e-8
    by the oracle's evaluation; on a sample of 24 systems (the largest and
    the smallest among them) the mask, the subsystem and the threshold equal
    the oracle's bit for bit and the solution is within 1e-6 of the oracle's
    FP64 one."""
    from paper_2001_01158_gb300.autotune import tune_batch
    ctx = lcg.Context(0)
    items = gen.cfg4_batch(seed=0)
    systems = [(d["op"].shape[0], d["op"].shape[1], cu(d["op"].D), cu(d["op"].Tx), cu(d["op"].Ty)) for d in items]
    batch = lcg.Batch(ctx, systems)
    b = cu(np.concatenate([d["b"] for d in items]))
    x0 = cu(np.concatenate([d["x0"] for d in items]))
    prm = lcg.batch_params(beta=1e-3, layers=2, tol=1e-8, inner_tol=1e-4)
    tune_batch(batch, b, x0, prm)
    x = x0.clone()
    batch.capture(b, x, prm)
    x.copy_(x0)
    batch.replay()
    torch.cuda.synchronize()
    st = batch.stats()
    xs = x.cpu().numpy()
    # the sample holds the largest and the smallest system
    sizes = [d["op"].n for d in items]
    sample = set(np.random.default_rng(1).choice(len(items), size=22, replace=False).tolist())
    sample |= {int(np.argmax(sizes)), int(np.argmin(sizes))}
    for s, d in enumerate(items):
        A = oracle.from_stencil(d["op"])
        xg = xs[batch.offsets[s]:batch.offsets[s + 1]]
        assert st[s]["status"] == 0 and oracle.relres(A, d["b"], xg) <= 1e-8, s
        if s in sample:
            m = oracle.mark_residual(A, d["b"], d["x0"], oracle.THR_REL_MAX, 1e-3, oracle.EXP_DILATE, 2)
            ex = oracle.extract(A, m["mask"], d["b"], d["x0"])
            assert st[s]["K"] == m["K"] and st[s]["nnzB"] == len(ex["B"].col) and st[s]["tau"] == m["tau"], s
            assert_domain_equal(batch, s, m, ex)
            xr, _, _, _ = oracle.pcg(A, d["b"], d["x0"], tol=1e-13)
            assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr), s
