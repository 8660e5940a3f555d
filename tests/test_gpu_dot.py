"""The reproducible dot product lc_op_dot (products summed exactly in 128-bit
fixed point): the sum of the FP64 products equals Python's
correctly rounded math.fsum bit for bit (products within 2^40 of the
largest), does not depend on the order of the terms, survives cancellation,
and propagates NaN."""
import math

import numpy as np
import pytest
import torch

import paper_2001_01158_gb300 as lcg

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def ctx():
    lcg.build()
    return lcg.Context(0)


def identity_op(ctx, n):
    rp = torch.arange(n + 1, dtype=torch.int32, device=DEV)
    ci = torch.arange(n, dtype=torch.int32, device=DEV)
    return lcg.CsrOperator(ctx, rp, ci, torch.ones(n, dtype=torch.float64, device=DEV))


def gdot(ctx, op, x, y):
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    lcg.dot(ctx, op, torch.as_tensor(x, device=DEV), torch.as_tensor(y, device=DEV), out)
    torch.cuda.synchronize()
    return float(out.item())


def bits(v):
    return np.array([v], dtype=np.float64).view(np.int64)[0]


@pytest.mark.parametrize("n", [1, 31, 1000, 65537, 1 << 22])
def test_dot_equals_fsum_bit_for_bit(ctx, n):
    rng = np.random.default_rng(n)
    x = rng.uniform(0.5, 2.0, n) * np.exp2(rng.integers(-8, 9, n)) * rng.choice([-1.0, 1.0], n)
    y = rng.uniform(0.5, 2.0, n) * np.exp2(rng.integers(-8, 9, n))
    op = identity_op(ctx, n)
    got = gdot(ctx, op, x, y)
    ref = math.fsum((x * y).tolist())
    assert bits(got) == bits(ref)
    # any order of the terms gives the same bits
    perm = rng.permutation(n)
    assert bits(gdot(ctx, op, x[perm], y[perm])) == bits(got)


def test_dot_cancellation_and_special_values(ctx):
    n = 4096
    op = identity_op(ctx, n)
    rng = np.random.default_rng(3)
    a = rng.uniform(1e6, 1e7, n // 2)
    x = np.concatenate([a, -a])
    x[7] += 3e-3   # survives the cancellation of the 1e6-sized terms
    y = np.ones(n)
    assert bits(gdot(ctx, op, x, y)) == bits(math.fsum(x.tolist()))
    assert gdot(ctx, op, np.zeros(n), np.ones(n)) == 0.0
    x2 = np.ones(n)
    x2[100] = np.nan
    assert math.isnan(gdot(ctx, op, x2, np.ones(n)))
    x3 = np.ones(n)
    x3[5] = np.inf
    assert math.isnan(gdot(ctx, op, x3, np.ones(n)))
