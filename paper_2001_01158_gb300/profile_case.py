"""One solve of the 2D moving-front workload, for profiler captures.

    python -m paper_2001_01158_gb300.profile_case --n 1024 --kind global

Solves system 1 (x0 = 0) with the global PCG to obtain x^1, then system 2
from x^1 with the requested method, and prints its statistics as JSON.
The global PCG kernel launch of interest is therefore the second one of
the process (ncu: -k regex:pcg_kernel -s 1 -c 1)."""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--kind", choices=["global", "alg1", "alg1_gradient"], default="global")
    a = ap.parse_args()
    import torch

    import gen
    import paper_2001_01158_gb300 as lcg

    lcg.build()
    dev = torch.device("cuda", 0)
    d = gen.cfg2_fronts2d(seed=0, n=a.n)
    op, seq = d["op"], d["seq"]
    T = lambda v: torch.as_tensor(v, dtype=torch.float64, device=dev)  # noqa: E731
    ctx = lcg.Context(0)
    gop = lcg.StencilOperator(ctx, op.shape, T(op.D), T(op.Tx), T(op.Ty))
    sp = lcg.SolveParams(1e-8, 200000, lcg.PREC_FP64, 0.0, 0)
    x1 = torch.zeros(op.n, dtype=torch.float64, device=dev)
    lcg.pcg_solve(ctx, gop, T(seq.source(1)), x1, sp)
    b2 = x1 / op.meta["dt"] + T(seq.source(2))
    x = x1.clone()
    st = lcg.Stats()
    if a.kind == "global":
        lcg.pcg_solve(ctx, gop, b2, x, sp, st)
    else:
        mode = lcg.MARK_RESIDUAL if a.kind == "alg1" else lcg.MARK_GRADIENT
        lcg.solve_local_then_global(ctx, gop, b2, x, lcg.default_params(mode, tol=1e-8), st)
    print(json.dumps({"n": a.n, "kind": a.kind, **st.as_dict()}))


if __name__ == "__main__":
    main()
