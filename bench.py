#!/usr/bin/env python3
"""Benchmark of the local character-based solve on one GB300 (or N replicas).

Workload (one "step" = one system of the sequence solved end to end by the
hot path): a 2048 x 2048 5-point backward-Euler diffusion operator with
discontinuous conductivity (background 1, 64 seeded rectangles, k
log-uniform in [1, 1e3]) and a Gaussian hot front (sigma = 30 cells) that
moves 8 cells per step over 20 steps.  System n is A x = x^{n-1}/dt + s^n,
started from the reference solution x^{n-1} (computed once, before timing,
by the global PCG of this library and kept resident in HBM).  Each step runs
Alg 1 with residual marking as the paper runs it (Sec. 2.3.1, Alg 3: tau =
eps ||b||_2 / sqrt(N) with eps = 1e-8, the solve's tolerance, and E_max = 1),
extraction, local Jacobi-PCG, assembly, the check of x~ and the warm-started
global Jacobi-PCG to relres 1e-8.  The same systems are also solved by plain
global Jacobi-PCG, by Alg 1 with gradient marking (Alg 2, alpha = 1e-4), with
the relative threshold 1e-3 max|r0| and 2 dilation layers, with one
Gauss-Seidel sweep, and in mixed precision, for comparison.

The JSON line reports time-to-solution per system (lower is better), the
roofline of the dominant kernel (the one with the largest share of the step),
the kernel count, SM clocks sampled during the timed region, an end-to-end
figure through the C ABI with host buffers, and the oracle timed on the host
cores.

`--impl reference` times the oracle (plain serial FP64 CPU code) instead.
"""
from __future__ import annotations

import argparse
import contextlib
import datetime
import hashlib
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-solution per system and SpMV HBM GB/s: local-first vs global PCG at relres 1e-8"
UNIT = "ms/system"
WORKLOAD = ("2D 2048x2048 5-point FP64 diffusion, 64 rectangles k in [1,1e3], Gaussian front sigma=30 moving "
            "8 cells/step, 20 backward-Euler steps; Alg 1 with residual marking (Alg 3: eps ||b||/sqrt(N), "
            "eps = 1e-8, E_max = 1), Jacobi-PCG to relres 1e-8")

# Alg 1 settings of the 2048^2 workload (keyword arguments of both the
# binding's default_params and the oracle's solve_local_then_global).
# Residual marking as the paper runs it (Sec. 2.3.1, Alg 3: eps = the
# solve's tolerance, E_max = 1); gradient marking (Alg 2) with the paper's
# alpha = 1e-4 and no further layers; and the relative threshold 1e-3 max|r0|
# with 2 dilation layers, the marking stated for the 128 x 128 case.
MARK_ALG3 = dict(mark_mode=0, thr_mode=0, thr_param=1e-8, exp_mode=2, exp_rounds=1)
MARK_REL = dict(mark_mode=0, thr_mode=1, thr_param=1e-3, exp_mode=1, exp_rounds=2)
MARK_GRAD = dict(mark_mode=1, alpha=1e-4, grad_layers=0)

# Algorithmic bytes of a Jacobi-PCG iteration on the 2D FP64 operator, per
# cell: set-up / true residual pass reads b, x, D, Tx, Ty, dinv and writes r, z
# (64 B); each iteration moves 120 B (phase A: z, p_old, D, Tx, Ty in, p, q
# out; phase B: x, p, r, q, dinv in, x, r, z out).  The kernel iterates on
# the symmetrically scaled system D^-1/2 A D^-1/2 (unit diagonal: no D, no
# dinv, z = r) and moves 92 B per cell and iteration (phase A: r, p_old, x,
# Tx, Ty in, p, q, x out -- x += alpha p_old rides on the p_old load; phase
# B: r, q in, fl32(D) for the FP32 stopping norm, r out); the roofline
# reports the algorithmic figure.
SETUP_BYTES = 64
ITER_BYTES = 120
IMPL_ITER_BYTES = 92
# FP64 instructions the scaled kernel issues per cell: 8 per iteration (phase
# A: 1 for p, 4 fma for q -- p.q runs on FP32 pairs; phase B: x, r, r.r),
# 10 per residual pass
DP_SETUP = 10
DP_ITER = 8
DP_PEAK_GOPS = 152 * 2 * 2.07   # FP64 FMA instructions per second, in G (nominal 1.25 TFLOP/s)
# Algorithmic bytes of a Jacobi-PCG iteration on a CSR matrix, per row and
# per entry: row pointers 4 B; phase A z, p_old in and p, q out (32 B) plus
# 12 B per entry (column index, value); phase B x, p, r, q, dinv in and x, r,
# z out (64 B) -- 100 B per row and 12 B per entry.
LOCAL_ROW_BYTES = 100
LOCAL_ENTRY_BYTES = 12
# FP64 instructions of the pipelined local solve per row and iteration
# besides the product's one per entry of B: the six vector updates (z, s, p,
# x^, r^, w); its sums run on FP32 pairs
LOCAL_DP_ROW_ITER = 6


def local_fp64_issue(per, t_s: float) -> dict:
    """The local solve seen from FP64 issue: (nnz(B) + 6 K) FP64 instructions
    per iteration over the solves' event time t_s (seconds), against the
    nominal FP64 rate."""
    dp = sum((s["nnzB"] + LOCAL_DP_ROW_ITER * s["K"]) * s["it_local"] for s in per)
    ach = dp / t_s / 1e9 if t_s > 0 else 0.0
    return {"bound": "alu", "achieved": ach, "peak": DP_PEAK_GOPS, "unit": "G FP64 instr/s",
            "frac": ach / DP_PEAK_GOPS, "alg_fp64_instr_per_row_iter": f"1 per entry of B + {LOCAL_DP_ROW_ITER}",
            "note": "the local solve kernel; neither this nor the HBM view is saturated: grid-barrier and L2 latency"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["lc", "reference"], default="lc")
    ap.add_argument("--side", "--n", dest="n", type=int, default=2048, help="grid side")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-system batched workload")
    ap.add_argument("--no-heat", action="store_true", help="skip the nonlinear heat runs (Sec. 3.2)")
    ap.add_argument("--profile-case", choices=PROFILE_CASES, default=None,
                    help="run one solve of a workload for a profiler capture and print its statistics (no timing)")
    ap.add_argument("--systems", type=int, default=512,
                    help="--profile-case batched: the first this many systems of the 512-system workload")
    return ap.parse_args()


# ----------------------------------------------------------------- utilities

def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", "0"))
        local = int(os.environ.get("LOCAL_RANK", str(rank)))
        gpu = args.impl == "lc" and torch.cuda.is_available()
        if gpu:
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if gpu else "gloo")
        return rank, ws, local
    return 0, 1, 0


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws, device=None):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms, each sample
    with nvidia-smi's own timestamp so that the summary keeps only the samples
    taken inside the timed window."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def __enter__(self):
        cmd = ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if shutil.which("stdbuf"):
            cmd = ["stdbuf", "-oL"] + cmd   # one line per sample, not one block per 4 KB
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
            return self
        t_end = time.monotonic() + 3.0          # nvidia-smi takes a moment to start sampling
        while not self.lines and time.monotonic() < t_end and self.proc.poll() is None:
            time.sleep(0.01)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self, t0: float, t1: float):
        """The timed window, as wall-clock seconds (time.time())."""
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.1)                     # the sample that closes the window
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm, mx = float(f[2]), float(f[3])
            except ValueError:
                continue
            rows.append((ts, sm, mx, [n for n, v in zip(names, f[6:10]) if v.lower().startswith("active")]))
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        where = "timed region" if self.window else "sampler lifetime"
        inside = rows
        if self.window:
            inside = [r for r in rows if self.window[0] <= r[0] <= self.window[1]]
            if not inside:   # a window shorter than the sampling period: the samples around it
                where = "warm-up and timed region"
                inside = rows
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted({n for r in inside for n in r[3]}), "samples": len(inside), "sampled": where,
                "window_ms": round((self.window[1] - self.window[0]) * 1e3, 1) if self.window else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


GLOBAL_SOURCES = ("lc_pcg_impl.cuh", "lc_pcg.cu", "lc_device.cuh")
LOCAL_SOURCES = ("lc_pcgpipe.cu", "lc_pcg_impl.cuh", "lc_device.cuh", "lc_internal.cuh")


def source_digest(names=GLOBAL_SOURCES) -> str:
    """Digest of a kernel's sources (default: the global PCG kernel's -- the
    kernels, the 2D launcher and the device header with its descriptors,
    barrier and reductions)."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2001_01158_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_cell_iter():
    """DRAM bytes per cell and iteration of the global PCG kernel from the
    committed ncu summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "pcg_stencil2d_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for ln in f:
            if "=" in ln and not ln.lstrip().startswith("#"):
                k, v = ln.split("=", 1)
                vals[k.strip()] = v.strip()
    if vals.get("pcg_sources_sha256_16") != source_digest():
        return None
    try:
        return float(vals["dram_bytes_per_cell_iter"]), float(vals.get("dram_bytes_per_cell_setup", "nan"))
    except (KeyError, ValueError):
        return None


def ncu_local_traffic(rows: float):
    """DRAM bytes per launch of the local solve kernel, given the launch's
    subsystem rows, from the committed ncu summary (bytes per row and launch:
    the subsystem is read into L2 once and stays there) if it was taken on
    the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "pcg_local_csr_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for ln in f:
            if "=" in ln and not ln.lstrip().startswith("#"):
                k, v = ln.split("=", 1)
                vals[k.strip()] = v.strip()
    if vals.get("pcg_sources_sha256_16") != source_digest(LOCAL_SOURCES):
        return None
    try:
        return float(vals["dram_bytes_per_row_launch"]) * rows
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------- oracle side

class OracleChain:
    """The bench workload solved by the oracle alone: system j (j = 0 .. 19)
    is A x = x^j/dt + s^{j+1} started from x^j, with x^0 = 0 and x^{j+1} the
    oracle's own Alg 1 solution of system j (relres 1e-8) -- the GPU arm's
    systems, with the oracle's chain of previous solutions instead of the
    library's (no input of the oracle comes from the CUDA path).  Step k
    solves system k mod 20; a system is solved only once its start exists,
    so steps run in order from k = 0."""

    def __init__(self, n: int, seed: int = 0):
        import numpy as np

        import gen
        import oracle
        d = gen.cfg2_fronts2d(seed=seed, n=n)
        self.A = oracle.from_stencil(d["op"])
        self.seq, self.dt, self.n = d["seq"], d["op"].meta["dt"], n
        self.states = {0: np.zeros(self.A.n)}

    def solve(self, k: int):
        """Alg 1 (the headline's residual marking, Alg 3; relres 1e-8) on
        system k mod 20; returns (seconds, stats)."""
        import oracle
        j = k % self.seq.steps
        x0 = self.states[j]
        b = x0 / self.dt + self.seq.source(j + 1)
        t = time.perf_counter()
        x, st, _ = oracle.solve_local_then_global(self.A, b, x0, **MARK_ALG3, tol=1e-8)
        dt = time.perf_counter() - t
        self.states.setdefault(j + 1, x)
        return dt, st


def oracle_legs(n: int, serial_steps: int, omp_steps: int, warmup: int = 0):
    """Times the oracle on the bench workload at n x n, both legs over the
    chain's steps k = 0, 1, ... (the first `warmup` untimed): the serial
    parity oracle (one thread) builds the chain over warmup + serial_steps
    steps; the timing-only OpenMP build (row loops on all host cores) then
    solves steps 0 .. warmup + omp_steps - 1 from the same chain states.
    Returns both legs (ms per system, threads, systems)."""
    import oracle
    from oracle.build import build_oracle
    build_oracle()
    build_oracle(openmp=True)
    ch = OracleChain(n)
    legs = {}
    for name, steps in (("serial", serial_steps), ("omp", omp_steps)):
        ms, systems = [], []
        with (oracle.openmp_build() if name == "omp" else contextlib.nullcontext()):
            threads = oracle.threads()
            for k in range(warmup + steps):
                dt, _ = ch.solve(k)
                if k >= warmup:
                    ms.append(dt * 1e3)
                    systems.append(k % ch.seq.steps)
        legs[name] = {"ms": ms, "threads": threads, "systems": systems}
    legs["chain"] = ch
    return legs


def run_reference(args, rank, ws):
    """The reference arm: the oracle on the host cores, on the GPU arm's
    workload (full n x n systems, the oracle's own chain of previous
    solutions): W untimed and K timed steps of the serial oracle (the value),
    and the same steps by its OpenMP build on all host cores beside it."""
    if rank != 0:
        return
    legs = oracle_legs(args.n, args.steps, args.steps, warmup=args.warmup)
    ser, omp = legs["serial"], legs["omp"]
    v = statistics.mean(ser["ms"]) if ser["ms"] else float("nan")
    sample = (f"serial oracle Alg 1 (plain FP64 C, 1 thread) on the full {args.n}x{args.n} systems "
              f"{ser['systems']} of the moving-front sequence, each from the oracle's own previous solution; "
              f"{args.warmup} untimed + {args.steps} timed steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("2048x2048", f"{args.n}x{args.n}"), "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": ser["threads"], "kind": "oracle", "sample": sample},
        "cpu_openmp": {"value": statistics.mean(omp["ms"]) if omp["ms"] else None, "unit": UNIT,
                       "cores": omp["threads"], "kind": "oracle",
                       "sample": (f"OpenMP build of the same oracle source (row loops on {omp['threads']} threads, "
                                  f"timing only) on the same systems {omp['systems']}")},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU side

def parse_cpulist(spec: str) -> set:
    """CPU numbers of a sysfs cpulist ("0-3,8,10-11")."""
    cpus = set()
    for part in spec.strip().split(","):
        if "-" in part:
            lo, hi = part.split("-")
            cpus.update(range(int(lo), int(hi) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def gpu_local_cpus(dev_index: int):
    """Bind this process to the host CPUs next to the GPU (its PCI device's
    local_cpulist, intersected with the CPUs the process may use), so that
    the pinned host buffers of the end-to-end loop are first touched on the
    GPU's own NUMA node.  Returns a short description, or None when the
    topology is not readable."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev_index)
        bus = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        base = f"/sys/bus/pci/devices/{bus}"
        with open(f"{base}/local_cpulist") as f:
            cpus = parse_cpulist(f.read())
        allowed = os.sched_getaffinity(0)
        inter = cpus & allowed
        node = "?"
        if os.path.exists(f"{base}/numa_node"):
            with open(f"{base}/numa_node") as f:
                node = f.read().strip()
        if inter and inter != allowed:
            os.sched_setaffinity(0, inter)
        return f"GPU {bus} NUMA node {node}: {len(inter) if inter else len(allowed)} of {len(allowed)} CPUs"
    except Exception:
        return None


def run_gpu(args, rank, ws, local):
    import numpy as np
    import torch

    import gen
    import paper_2001_01158_gb300 as lcg

    lcg.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    d = gen.cfg2_fronts2d(seed=rank, n=args.n)
    op, seq = d["op"], d["seq"]
    N = op.n
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
    ctx = lcg.Context(local)
    gop = lcg.StencilOperator(ctx, op.shape, T(op.D), T(op.Tx), T(op.Ty))
    sp = lcg.SolveParams(1e-8, 200000, lcg.PREC_FP64, 0.0, 0)

    # the sequence's reference states, resident in HBM
    nsys = seq.steps
    xs = [torch.zeros(N, dtype=torch.float64, device=dev)]
    bs = []
    for k in range(1, nsys + 1):
        b = xs[-1] / op.meta["dt"] + T(seq.source(k))
        x = xs[-1].clone()
        lcg.pcg_solve(ctx, gop, b, x, sp)
        bs.append(b)
        xs.append(x)
    torch.cuda.synchronize(dev)

    prm_res = lcg.default_params(**MARK_ALG3, tol=1e-8)
    prm_rel = lcg.default_params(**MARK_REL, tol=1e-8)
    prm_grad = lcg.default_params(**MARK_GRAD, tol=1e-8)
    # inner_tol 1e-3: the pipelined FP32 inner solve's recurrences drift past
    # a ~1e-3 reduction, so deeper inner solves only add iterations
    prm_mixed = lcg.default_params(**MARK_ALG3, tol=1e-8, precision=lcg.PREC_MIXED, inner_tol=1e-3)
    # Alg 1 with its step-7 smoothing: one red-black Gauss-Seidel sweep, as in the paper's runs
    prm_gs = lcg.default_params(**MARK_ALG3, tol=1e-8, gs_sweeps=1)
    prms = {"res": prm_res, "rel": prm_rel, "grad": prm_grad, "mixed": prm_mixed, "gs": prm_gs}
    sp_mixed = lcg.SolveParams(1e-8, 200000, lcg.PREC_MIXED, 1e-4, 30)
    work = torch.empty(N, dtype=torch.float64, device=dev)

    def system(k):
        j = k % nsys
        return bs[j], xs[j]

    def solve(kind, k, stats):
        b, x0 = system(k)
        work.copy_(x0, non_blocking=True)
        if kind == "global":
            lcg.pcg_solve(ctx, gop, b, work, sp, stats)
        elif kind == "global_mixed":
            lcg.pcg_solve(ctx, gop, b, work, sp_mixed, stats)
        else:
            lcg.solve_local_then_global(ctx, gop, b, work, prms[kind], stats)

    def timed_loop(kind, steps, warmup, clocks=None):
        st = lcg.Stats()
        for k in range(warmup):
            solve(kind, k, st)
        torch.cuda.synchronize(dev)
        barrier(ws)
        per = []
        launches0 = lcg.kernel_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        e0.record(stream)
        for k in range(steps):
            solve(kind, warmup + k, st)
            per.append(st.as_dict())
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if clocks is not None:
            clocks.mark(w0, time.time())
        barrier(ws)
        launches = lcg.kernel_launch_count() - launches0
        ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
        return ms, per, launches

    with ClockSampler(local) as cs:
        ms_res, per_res, launches = timed_loop("res", args.steps, args.warmup, cs)
    clocks = cs.summary()
    ms_glob, per_glob, _ = timed_loop("global", args.steps, args.warmup)
    ms_grad, per_grad, _ = timed_loop("grad", args.steps, args.warmup)
    ms_rel, per_rel, _ = timed_loop("rel", args.steps, args.warmup)
    ms_gs, per_gs, _ = timed_loop("gs", args.steps, args.warmup)
    ms_mixed, per_mixed, _ = timed_loop("mixed", args.steps, args.warmup)
    ms_gmixed, per_gmixed, _ = timed_loop("global_mixed", args.steps, args.warmup)
    # system 0 (b = s^1, x0 = 0) by mixed precision and by FP64 Alg 1, kept
    # for the comparison with the oracle's FP64 solution (rank 0, below)
    solve("mixed", 0, lcg.Stats())
    x_mixed0 = work.cpu().numpy()
    solve("res", 0, lcg.Stats())
    x_res0 = work.cpu().numpy()

    # rooflines, each over CUDA-event times the library records on the
    # launching stream.  The global PCG kernel: the plain global solves
    # (every launch a full solve from x^{n-1}).
    def pcg_bytes(s):
        checks = 1 + (0 if s["early_exit"] else 1 + s["restarts"])
        return N * (SETUP_BYTES * checks + ITER_BYTES * s["it_global"])

    peak, peak_kind = measured_peaks()
    byts_g = sum(pcg_bytes(s) for s in per_glob)
    t_g = sum(s["t_global_ms"] for s in per_glob) * 1e-3
    gbs_global = byts_g / t_g / 1e9 if t_g > 0 else 0.0
    tr = ncu_traffic_per_cell_iter()
    mean_it_g = statistics.mean(s["it_global"] for s in per_glob)
    traffic_g = None
    if tr is not None:
        bpc_iter, bpc_setup = tr
        traffic_g = float(N * (bpc_iter * mean_it_g + (bpc_setup if math.isfinite(bpc_setup) else SETUP_BYTES) * 2))
    # the same kernel seen from FP64 issue (DP_ITER, DP_SETUP); peak = 152 SMs
    # x 2 FP64 FMA/clk x 2.07 GHz (the nominal 1.25 TFLOP/s)
    dp = sum(N * (DP_SETUP * (2 + s["restarts"]) + DP_ITER * s["it_global"]) for s in per_glob)
    dp_achieved = dp / t_g / 1e9 if t_g > 0 else 0.0
    roof_global = {"bound": "hbm", "achieved": gbs_global, "peak": peak, "unit": "GB/s", "frac": gbs_global / peak,
                   "traffic": traffic_g,
                   "kernel": "pcg_kernel<Op2DW<double,4,true,true,true>> "
                             "(global Jacobi-PCG on D^-1/2 A D^-1/2, FP64 vectors)",
                   "peak_source": f"{peak_kind} hbm_gbs", "alg_bytes_per_cell_iter": ITER_BYTES,
                   "impl_bytes_per_cell_iter": IMPL_ITER_BYTES}
    # The local solve inside Alg 1: Jacobi-PCG on the extracted CSR
    # subsystem B (K rows, nnz(B) entries), algorithmic LOCAL_ROW_BYTES per
    # row and LOCAL_ENTRY_BYTES per entry and iteration, over the local
    # solve's event time.
    byts_l = sum(s["K"] * LOCAL_ROW_BYTES * s["it_local"] + s["nnzB"] * LOCAL_ENTRY_BYTES * s["it_local"]
                 for s in per_res)
    t_l = sum(s["t_local_ms"] for s in per_res) * 1e-3
    gbs_local = byts_l / t_l / 1e9 if t_l > 0 else 0.0
    roof_local = {"bound": "hbm", "achieved": gbs_local, "peak": peak, "unit": "GB/s", "frac": gbs_local / peak,
                  "traffic": ncu_local_traffic(statistics.mean(s["K"] for s in per_res)),
                  "kernel": "pcgpipe_kernel (local Jacobi-PCG on the extracted subsystem: pipelined CG on "
                            "diag(B)^-1/2 B diag(B)^-1/2)",
                  "peak_source": f"{peak_kind} hbm_gbs", "alg_bytes_per_row_iter": LOCAL_ROW_BYTES,
                  "alg_bytes_per_entry_iter": LOCAL_ENTRY_BYTES,
                  "note": "FP64 issue and latency: one grid barrier per iteration; B and the vectors stay in L2"}
    t_glob_in_alg1 = sum(s["t_global_ms"] for s in per_res) * 1e-3
    dominant = "local_solve" if t_l >= t_glob_in_alg1 else "global_pcg"
    if dominant == "global_pcg":   # the global kernel's figures over its launches inside Alg 1
        byts = sum(pcg_bytes(s) for s in per_res)
        ach = byts / t_glob_in_alg1 / 1e9 if t_glob_in_alg1 > 0 else 0.0
        roofline = dict(roof_global, achieved=ach, frac=ach / peak, traffic=None)
    else:
        roofline = dict(roof_local)
    roofline["dominant"] = dominant
    roofline["share_of_step"] = max(t_l, t_glob_in_alg1) / (ms_res * 1e-3)
    mean_it = statistics.mean(s["it_global"] for s in per_res)

    # end to end through the C ABI with host buffers: every system's b and x0
    # come from pinned host memory and its solution goes back to it.  The
    # copies run on their own stream, overlapped with the neighbouring
    # systems' solves (inputs double-buffered on the device), as a serving
    # loop would run them; each step's copies and solve are all inside the
    # timed region.
    cpus0 = os.sched_getaffinity(0)
    affinity = gpu_local_cpus(local)
    b_h = [bs[j].cpu().pin_memory() for j in range(nsys)]
    x_h = [xs[j].cpu().pin_memory() for j in range(nsys)]
    out_h = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(2)]
    b_d = [torch.empty(N, dtype=torch.float64, device=dev) for _ in range(2)]
    x_d = [torch.empty(N, dtype=torch.float64, device=dev) for _ in range(2)]
    cstream = torch.cuda.Stream(dev)
    h2d_done = [torch.cuda.Event() for _ in range(2)]
    solved = [torch.cuda.Event() for _ in range(2)]
    st = lcg.Stats()

    def h2d(k):
        j, s = k % nsys, k % 2
        with torch.cuda.stream(cstream):
            b_d[s].copy_(b_h[j], non_blocking=True)
            x_d[s].copy_(x_h[j], non_blocking=True)
            h2d_done[s].record(cstream)

    def e2e_run(k0, steps):
        # buffer s = k % 2 is rewritten by h2d(k + 2), issued after the
        # copy-back of step k on the same (in-order) copy stream
        h2d(k0)
        for k in range(k0, k0 + steps):
            s = k % 2
            if k + 1 < k0 + steps:
                h2d(k + 1)   # the next system's inputs while this one solves
            stream.wait_event(h2d_done[s])
            lcg.solve_local_then_global(ctx, gop, b_d[s], x_d[s], prm_res, st, stream=stream)
            solved[s].record(stream)
            with torch.cuda.stream(cstream):
                cstream.wait_event(solved[s])
                out_h[s].copy_(x_d[s], non_blocking=True)
        torch.cuda.synchronize(dev)

    e2e_run(0, args.warmup)
    barrier(ws)
    t0 = time.perf_counter()
    e2e_run(args.warmup, args.steps)
    barrier(ws)
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, ws, dev)
    os.sched_setaffinity(0, cpus0)   # the oracle's legs below use every CPU again

    total_sys = args.steps * ws
    value = ms_res / total_sys
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_res / args.steps, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("2048x2048", f"{args.n}x{args.n}"), "N": N,
                   "systems": nsys, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (operator + 20 resident systems + PCG vectors > 1 GB)"},
        "roofline": roofline,
        "roofline_local_solve": roof_local,
        "roofline_local_solve_fp64_issue": local_fp64_issue(per_res, t_l),
        "roofline_global_pcg": roof_global,
        "roofline_global_pcg_fp64_issue": {
            "bound": "alu", "achieved": dp_achieved, "peak": DP_PEAK_GOPS, "unit": "G FP64 instr/s",
            "frac": dp_achieved / DP_PEAK_GOPS, "alg_fp64_instr_per_cell_iter": DP_ITER,
            "note": "the global kernel; ncu shows its FP64 pipe ~71% busy at ~57% DRAM throughput"},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": e2e_ms / total_sys, "unit": UNIT, "host_cpus": affinity, "h2d_bytes_per_step": 2 * 8 * N,
                "d2h_bytes_per_step": 8 * N},
        "global_pcg": {"value": ms_glob / total_sys, "unit": UNIT,
                       "iterations": statistics.mean(s["it_global"] for s in per_glob), "hbm_gbs": gbs_global},
        "local_first_residual": {
            "value": value, "marking": "Alg 3: tau = eps ||b||/sqrt(N), eps = 1e-8, E_max = 1",
            "K": statistics.mean(s["K"] for s in per_res), "nnzB": statistics.mean(s["nnzB"] for s in per_res),
            "eta": statistics.mean(s["eta"] for s in per_res),
            "it_local": statistics.mean(s["it_local"] for s in per_res),
            "it_global": mean_it, "early_exit_frac": statistics.mean(s["early_exit"] for s in per_res),
            "t_mark_ms": statistics.mean(s["t_mark_ms"] for s in per_res),
            "t_extract_ms": statistics.mean(s["t_extract_ms"] for s in per_res),
            "t_local_ms": statistics.mean(s["t_local_ms"] for s in per_res),
            "t_global_ms": statistics.mean(s["t_global_ms"] for s in per_res),
            "relres_max": max(s["relres_final"] for s in per_res)},
        "local_first_relative_threshold": {
            "value": ms_rel / total_sys, "marking": "tau = 1e-3 max|r0|, 2 dilation layers",
            "eta": statistics.mean(s["eta"] for s in per_rel),
            "it_local": statistics.mean(s["it_local"] for s in per_rel),
            "it_global": statistics.mean(s["it_global"] for s in per_rel),
            "t_local_ms": statistics.mean(s["t_local_ms"] for s in per_rel),
            "t_global_ms": statistics.mean(s["t_global_ms"] for s in per_rel),
            "relres_max": max(s["relres_final"] for s in per_rel)},
        "local_first_gs1": {
            "value": ms_gs / total_sys, "gs_sweeps": 1,
            "it_global": statistics.mean(s["it_global"] for s in per_gs),
            "early_exit_frac": statistics.mean(s["early_exit"] for s in per_gs),
            "relres_tilde": statistics.mean(s["relres_tilde"] for s in per_gs),
            "relres_max": max(s["relres_final"] for s in per_gs)},
        "local_first_gradient": {
            "value": ms_grad / total_sys, "marking": "Alg 2: alpha = 1e-4",
            "eta": statistics.mean(s["eta"] for s in per_grad),
            "it_local": statistics.mean(s["it_local"] for s in per_grad),
            "it_global": statistics.mean(s["it_global"] for s in per_grad),
            "relres_max": max(s["relres_final"] for s in per_grad)},
        "local_first_mixed_precision": {
            "value": ms_mixed / total_sys, "inner_tol": 1e-3,
            "inner_iterations": statistics.mean(s["it_global"] for s in per_mixed),
            "refinement_sweeps": statistics.mean(s["restarts"] for s in per_mixed),
            "relres_max": max(s["relres_final"] for s in per_mixed)},
        "global_pcg_mixed_precision": {
            "value": ms_gmixed / total_sys, "unit": UNIT, "inner_tol": 1e-4,
            "inner_iterations": statistics.mean(s["it_global"] for s in per_gmixed),
            "refinement_sweeps": statistics.mean(s["restarts"] for s in per_gmixed),
            "relres_max": max(s["relres_final"] for s in per_gmixed),
            # the FP32 inner CG inside the refinement: algorithmic 60 B per cell
            # and inner iteration (FP32 Jacobi-PCG; the scaled kernel moves 52
            # B), FP64 residual passes at 48 B per cell and sweep, over the
            # launch's CUDA-event time
            "roofline": {
                "bound": "hbm", "unit": "GB/s", "peak": peak,
                "achieved": sum(N * (60 * s["it_global"] + 48 * (1 + s["restarts"])) for s in per_gmixed) /
                (sum(s["t_global_ms"] for s in per_gmixed) * 1e-3) / 1e9,
                "frac": sum(N * (60 * s["it_global"] + 48 * (1 + s["restarts"])) for s in per_gmixed) /
                (sum(s["t_global_ms"] for s in per_gmixed) * 1e-3) / 1e9 / peak,
                "kernel": "ir_kernel<Op2DW<double,2>, Op2DW<float,4,true>>"}},
        "speedup_vs_global_pcg": ms_glob / ms_res,
        "speedup_relative_threshold_vs_global_pcg": ms_glob / ms_rel,
        "speedup_gradient_vs_global_pcg": ms_glob / ms_grad,
        "speedup_mixed_vs_global_pcg": ms_glob / ms_mixed,
        "speedup_global_mixed_vs_global_pcg": ms_glob / ms_gmixed,
    }
    if not args.no_batched:
        res["batched_512"] = run_batched(args, rank, dev, ws)
    if not args.no_batched:
        res["multigroup_64"] = run_multigroup(args, dev)
        res["batched_8_largest"] = run_batched_largest(args, dev)
    if not args.no_batched:
        res["csr_3t_1024"] = run_csr3t(dev, 1024)
        res["aniso3d_256"] = run_aniso3d(dev, 256)
    if not args.no_heat:
        res["heat_e1"] = {"99x99_100_steps": run_heat(dev, 99, 100), "1024x1024_10_steps": run_heat(dev, 1024, 10)}
    if rank == 0 and not args.no_cpu_baseline:
        # the error of the mixed-precision and FP64 results of system 0
        # against the serial oracle's FP64 Jacobi-PCG solution (relres 1e-12)
        import numpy as np

        import oracle
        from oracle.build import build_oracle
        build_oracle()
        A0 = oracle.from_stencil(op)
        x_o, st_o, it_o, rr_o = oracle.pcg(A0, seq.source(1), np.zeros(N), tol=1e-12)
        n_o = float(np.linalg.norm(x_o))
        res["local_first_mixed_precision"]["err_vs_fp64_oracle"] = float(np.linalg.norm(x_mixed0 - x_o)) / n_o
        res["local_first_residual"]["err_vs_fp64_oracle"] = float(np.linalg.norm(x_res0 - x_o)) / n_o
        res["oracle_reference_solution"] = {
            "system": 0, "solver": "serial oracle Jacobi-PCG from x0 = 0", "relres": rr_o, "iterations": it_o,
            "status": st_o}
        if "aniso3d_256" in res:
            aniso3d_errors(res["aniso3d_256"])
        # a bounded sample (about 15 s of serial CPU work): the serial oracle on
        # the chain's 20 systems, the OpenMP build on the same systems
        legs = oracle_legs(args.n, 20, 20)
        ser, omp = legs["serial"], legs["omp"]
        res["cpu_baseline"] = {
            "value": statistics.mean(ser["ms"]), "unit": UNIT, "cores": ser["threads"], "kind": "oracle",
            "sample": (f"serial oracle Alg 1 (plain FP64 C, 1 thread) on the full {args.n}x{args.n} systems "
                       f"{ser['systems']} of the same sequence, each from the oracle's own previous solution"),
            "openmp": {"value": statistics.mean(omp["ms"]), "cores": omp["threads"],
                       "sample": (f"OpenMP build of the same oracle source (timing only) on systems "
                                  f"{omp['systems']}")}}
    if "aniso3d_256" in res:
        res["aniso3d_256"].pop("_x", None)
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_heat(dev, n, steps):
    """The paper's nonlinear 2D heat test (Sec. 3.2: kappa = T^3.5, T = 1 / 1e-4 at
    x = 0 / 1, no flux in y, dt = 1e-2, T0 = exp(-100 x) + 1e-4, Picard to
    ||dT|| < 1e-8, linear tolerance 1e-10) on n x n cells for `steps` steps,
    by the global PCG, Alg 1 with gradient marking (alpha = 1e-4) and Alg 1
    with the paper's residual marking (eps ||b||/sqrt(N), E_max = 1).  Times
    are CUDA-event sums over all linear solves (the paper's CPU_total) and
    over whole steps (with assembly and the Picard update norms)."""
    import numpy as np
    import torch

    import paper_2001_01158_gb300 as lcg

    ctx = lcg.Context(dev.index)
    xc = (np.arange(n) + 0.5) / n
    T0 = torch.as_tensor(np.tile(np.exp(-100.0 * xc) + 1e-4, n), dtype=torch.float64, device=dev)
    bt, bv = [lcg.BC_DIRICHLET, lcg.BC_DIRICHLET, lcg.BC_NEUMANN, lcg.BC_NEUMANN], [1.0, 1e-4, 0.0, 0.0]
    D, Tx, Ty, b = (torch.empty(n * n, dtype=torch.float64, device=dev) for _ in range(4))
    work = torch.empty(2 * n * n, dtype=torch.float64, device=dev)
    lcg.heat2d_assemble(ctx, (n, n), 1.0 / n, 1e-2, bt, bv, T0 ** 3.5, T0, D, Tx, Ty, b)
    op = lcg.StencilOperator(ctx, (n, n, 1), D, Tx, Ty)
    methods = {
        "global": (0, lcg.default_params(tol=1e-10)),
        "gradient": (1, lcg.default_params(lcg.MARK_GRADIENT, alpha=1e-4, grad_layers=0, tol=1e-10)),
        "residual": (1, lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_EPS_NORMB, 1e-10, lcg.EXP_PAPER, 1, tol=1e-10)),
    }
    out, finals = {}, {}
    for name, (method, prm) in methods.items():
        hp = lcg.heat_params(1.0 / n, 1e-2, 3.5, bt, bv, method=method, params=prm)
        T = T0.clone()
        Tn = torch.empty_like(T)
        solve_ms = total_ms = 0.0
        pic = lin = K = 0
        for _ in range(steps):
            Tn.copy_(T)
            st = lcg.heat2d_step(ctx, op, hp, Tn, T, D, Tx, Ty, b, work)
            solve_ms += st.t_solve_ms
            total_ms += st.t_total_ms
            pic += st.picard_its
            lin += st.it_local + st.it_global
            K += st.K_sum
        finals[name] = T
        out[name] = {"linear_solve_ms": solve_ms, "step_ms": total_ms, "systems": pic, "cg_iterations": lin,
                     "eta_mean": K / max(1, pic) / (n * n)}
    for name in ("gradient", "residual"):
        out[name]["speedup_vs_global"] = out["global"]["linear_solve_ms"] / out[name]["linear_solve_ms"]
        out[name]["rel_diff_vs_global"] = float(torch.linalg.norm(finals[name] - finals["global"]) /
                                                torch.linalg.norm(finals["global"]))
    return out


def run_batched(args, rank, dev, ws):
    """512 independent 2D systems (sides log-uniform in [64, 512], local
    sources covering 1-30 % of cells): all of Alg 1 in one autotuned,
    graph-captured launch (FP32 inner CG, FP64 refinement, relres 1e-8),
    against the same systems solved one after another by global FP64 PCG."""
    import gen
    return batched_items(gen.cfg4_batch(seed=rank), dev, max(3, min(args.steps, 10)))


def run_csr3t(dev, n):
    """A 3T-like coupled system (three interleaved temperatures per cell of an
    n x n grid, 9-point diffusion each, 3 x 3 cell coupling; 3 n^2 unknowns)
    through the general CSR path: Alg 1 (residual marking) against the global
    Jacobi-PCG from the same start, and the CSR PCG kernel's algorithmic HBM
    rate (per row and iteration: row pointer 4 B + 12 B per entry + z, p_old
    in and p, q out 32 B + phase B 64 B)."""
    import numpy as np
    import torch

    import gen
    import paper_2001_01158_gb300 as lcg

    rp, ci, av = gen.threeT_2d(11, n, n)
    nrows, nnz = len(rp) - 1, len(ci)
    rng = np.random.default_rng(5)
    x0 = 1.0 + 0.1 * rng.standard_normal(nrows)
    s = np.zeros(nrows)
    c = rng.integers(n // 4, 3 * n // 4, size=2)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    disc = (((xx - c[0]) ** 2 + (yy - c[1]) ** 2) <= (n / 40.0) ** 2).ravel()
    s[3 * np.flatnonzero(disc)] = 1.0   # radiation source in a disc
    b = gen.csr_matvec(rp, ci, av, x0) + s
    T = lambda a, dt=torch.float64: torch.as_tensor(a, dtype=dt, device=dev)  # noqa: E731
    ctx = lcg.Context(dev.index)
    op = lcg.CsrOperator(ctx, T(rp, torch.int32), T(ci, torch.int32), T(av))
    bd, x0d = T(b), T(x0)
    sp = lcg.SolveParams(1e-8, 200000, lcg.PREC_FP64, 0.0, 0)
    prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2, tol=1e-8)
    out = {}
    for name, run in (("global", lambda x, st: lcg.pcg_solve(ctx, op, bd, x, sp, st)),
                      ("alg1", lambda x, st: lcg.solve_local_then_global(ctx, op, bd, x, prm, st))):
        st = lcg.Stats()
        run(x0d.clone(), st)   # warm-up
        times, its = [], []
        for _ in range(3):
            x = x0d.clone()
            run(x, st)
            times.append(st.t_total_ms)
            its.append((st.it_local, st.it_global, st.K, st.t_global_ms))
        out[name] = {"ms": statistics.median(times), "it_local": its[-1][0], "it_global": its[-1][1],
                     "K": its[-1][2]}
        if name == "global":
            byts = nrows * 100 + 12 * nnz
            out[name]["pcg_alg_GBs"] = byts * its[-1][1] / (its[-1][3] * 1e-3) / 1e9
    out["rows"], out["nnz"] = nrows, nnz
    out["speedup_alg1_vs_global"] = out["global"]["ms"] / out["alg1"]["ms"]
    return out


def run_aniso3d(dev, n):
    """The 3D anisotropic workload (n^3 cells, k ratios 1:10:100 with a
    lognormal perturbation, a source box): global FP64 Jacobi-PCG and Alg 1
    with FP32 inner CG + FP64 refinement, both to relres 1e-10, the mixed
    result's difference from the FP64 one, and each global solve's algorithmic
    HBM rate (FP64 128 B, FP32 inner 64 B per cell and iteration)."""
    import numpy as np
    import torch

    import gen
    import paper_2001_01158_gb300 as lcg

    d = gen.cfg3_aniso3d(seed=0, n=n)
    op = d["op"]
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
    ctx = lcg.Context(dev.index)
    gop = lcg.StencilOperator(ctx, op.shape, T(op.D), T(op.Tx), T(op.Ty), T(op.Tz))
    b, x0 = T(d["b"]), T(d["x0"])
    N = op.n
    sp = lcg.SolveParams(1e-10, 200000, lcg.PREC_FP64, 0.0, 0)
    prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2, tol=1e-10,
                             precision=lcg.PREC_MIXED, inner_tol=1e-5)
    out = {}
    st = lcg.Stats()
    x64 = x0.clone()
    lcg.pcg_solve(ctx, gop, b, x64.clone(), sp, st)   # warm-up
    x64 = x0.clone()
    lcg.pcg_solve(ctx, gop, b, x64, sp, st)
    out["global_fp64"] = {"ms": st.t_total_ms, "iterations": st.it_global,
                          "alg_GBs": N * 128 * st.it_global / (st.t_global_ms * 1e-3) / 1e9}
    xm = x0.clone()
    lcg.solve_local_then_global(ctx, gop, b, xm.clone(), prm, st)   # warm-up
    xm = x0.clone()
    lcg.solve_local_then_global(ctx, gop, b, xm, prm, st)
    out["alg1_mixed"] = {"ms": st.t_total_ms, "K": st.K, "inner_iterations": st.it_global,
                         "relres": st.relres_final,
                         "global_alg_GBs": N * 64 * st.it_global / (st.t_global_ms * 1e-3) / 1e9}
    out["speedup_mixed_vs_fp64"] = out["global_fp64"]["ms"] / out["alg1_mixed"]["ms"]
    # the solutions, for the comparison with the oracle's FP64 solution (rank 0)
    out["_x"] = {"problem": d, "fp64": x64.cpu().numpy(), "mixed": xm.cpu().numpy()}
    return out


def aniso3d_errors(out):
    """Errors of the 3D FP64 and mixed-precision solutions against the serial
    oracle's FP64 Jacobi-PCG solution of the same system (relres 1e-10)."""
    import numpy as np

    import oracle
    xs = out.pop("_x")
    d = xs["problem"]
    A = oracle.from_stencil(d["op"])
    x_o, st_o, it_o, rr_o = oracle.pcg(A, d["b"], d["x0"], tol=1e-10)
    n_o = float(np.linalg.norm(x_o))
    out["global_fp64"]["err_vs_fp64_oracle"] = float(np.linalg.norm(xs["fp64"] - x_o)) / n_o
    out["alg1_mixed"]["err_vs_fp64_oracle"] = float(np.linalg.norm(xs["mixed"] - x_o)) / n_o
    out["oracle_reference_solution"] = {"solver": "serial oracle Jacobi-PCG from x0", "relres": rr_o,
                                        "iterations": it_o, "status": st_o}


def run_batched_largest(args, dev):
    """The 8 largest systems of the 512-system workload (sides 500..512) as a
    batch of their own: a batch whose time is one large system's, where the
    autotuner's thread-block clusters (several SMs per system) pay."""
    import numpy as np

    import gen
    items = gen.cfg4_batch(seed=0)
    big = np.argsort([-d["op"].n for d in items])[:8]
    return batched_items([items[i] for i in big], dev, max(3, min(args.steps, 10)))


def run_multigroup(args, dev):
    """Multi-group stand-in (64 group systems on one 88 x 80 mesh with a
    shared pattern, Sec. 3.3's structure): one source iteration's 64 solves
    batched in one launch, against sequential FP64 Alg 1 and sequential
    global FP64 PCG."""
    import gen
    return batched_items(gen.mg_standin(seed=0), dev, max(3, min(args.steps, 10)), seq_alg1=True)


def batched_roofline(stats, ms):
    """Algorithmic bytes of one batched launch over its time.  Per system of
    n cells, K local rows, nnz(B) entries: marking 48 B (residual) + 9 B
    (threshold and two layers) + 5 B (compaction) per cell, 130 B per local
    row (gather); the local refinement: 60 B per row plus 8 B per entry of B
    per FP32 inner iteration, 32 B per row plus 12 B per entry per FP64
    residual sweep (two sweeps assumed); the global refinement: 60 B per cell
    per FP32 inner iteration (FP32 Jacobi-PCG on the stencil), 48 B per cell
    per FP64 residual pass (sweeps + 1) and 16 B per cell per x update."""
    byts = 0.0
    for s in stats:
        n, K, nz = s["n"], s["K"], s["nnzB"]
        sweeps = s["restarts"]
        byts += n * (48 + 9 + 5) + 130 * K
        byts += s["it_local"] * (60 * K + 8 * nz) + 2 * (32 * K + 12 * nz)
        byts += n * (60 * s["it_global"] + 48 * (sweeps + 1) + 16 * sweeps)
    peak, kind = measured_peaks()
    achieved = byts / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "alg_bytes": byts, "peak_source": f"{kind} hbm_gbs", "kernel": "batched_kernel (whole batch, one launch)"}


def batched_items(items, dev, reps, seq_alg1=False):
    import numpy as np
    import torch

    import paper_2001_01158_gb300 as lcg
    from paper_2001_01158_gb300.autotune import tune_batch

    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
    ctx = lcg.Context(dev.index)
    systems = [(d["op"].shape[0], d["op"].shape[1], T(d["op"].D), T(d["op"].Tx), T(d["op"].Ty)) for d in items]
    batch = lcg.Batch(ctx, systems)
    b = T(np.concatenate([d["b"] for d in items]))
    x0 = T(np.concatenate([d["x0"] for d in items]))
    prm = lcg.batch_params(beta=1e-3, layers=2, tol=1e-8, inner_tol=1e-4)
    cfg = tune_batch(batch, b, x0, prm)
    x = x0.clone()
    batch.capture(b, x, prm)
    for _ in range(2):
        x.copy_(x0)
        batch.replay()
    torch.cuda.synchronize(dev)
    ts = []
    for _ in range(reps):
        x.copy_(x0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.replay()
        e1.record()
        torch.cuda.synchronize(dev)
        ts.append(e0.elapsed_time(e1))
    st = batch.stats()
    ms_batched = statistics.median(ts)
    ops = [lcg.StencilOperator(ctx, (s[0], s[1], 1), s[2], s[3], s[4]) for s in systems]
    xs = [T(d["x0"]) for d in items]
    bs = [T(d["b"]) for d in items]

    def sequential(solve):
        for op_, b_, x_ in zip(ops[:8], bs[:8], xs[:8]):   # warm-up
            solve(op_, b_, x_.clone())
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for op_, b_, x_ in zip(ops, bs, xs):
            solve(op_, b_, x_.clone())
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    # the same systems, one at a time, by the global FP64 PCG (and by FP64 Alg 1)
    sp = lcg.SolveParams(1e-8, 200000, lcg.PREC_FP64, 0.0, 0)
    ms_seq = sequential(lambda o, bb, xx: lcg.pcg_solve(ctx, o, bb, xx, sp))
    cells = batch.cells
    out = {"systems": batch.nsys, "cells": cells, "ms_per_batch": ms_batched,
           "ms_per_system": ms_batched / batch.nsys, "cells_per_s": cells / (ms_batched * 1e-3),
           "sequential_global_fp64_ms": ms_seq, "speedup_vs_sequential_global_fp64": ms_seq / ms_batched,
           "eta_mean": statistics.mean(s["eta"] for s in st),
           "relres_max": max(s["relres_final"] for s in st), "all_converged": all(s["status"] == 0 for s in st),
           "inner_iterations_mean": statistics.mean(s["it_global"] for s in st),
           "autotuned": {k: cfg[k] for k in ("block", "ctas_per_sm", "cluster", "big_cells")},
           "roofline": batched_roofline(st, ms_batched),
           "launch": "one persistent kernel, CUDA-graph replay"}
    if seq_alg1:
        prm64 = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2, tol=1e-8)
        ms_a = sequential(lambda o, bb, xx: lcg.solve_local_then_global(ctx, o, bb, xx, prm64))
        out["sequential_alg1_fp64_ms"] = ms_a
        out["speedup_vs_sequential_alg1_fp64"] = ms_a / ms_batched
    return out


PROFILE_CASES = ["global2d", "alg1", "alg1_rel", "alg1_gradient", "alg1_steps", "mixed2d", "fp64_3d", "mixed3d", "csr3t", "batched", "heat"]


def profile_case(args):
    """One solve of a workload, for ncu captures (`--side` sets the grid side).

    2D cases: the moving-front system 2 from x^1 (x^1 is solved first by the
    global PCG, so the launch of interest is the second pcg_kernel / ir_kernel
    launch of the process: ncu -k regex:<kernel> -s 1 -c 1): global2d the
    global FP64 PCG, mixed2d the mixed-precision global solve, alg1 Alg 1 with
    the paper's residual marking (Alg 3), alg1_rel with the relative
    threshold and 2 layers, alg1_gradient with gradient marking (Alg 2);
    alg1_steps the bench's timed step, Alg 1 with the headline marking on
    systems 1 .. --systems of the sequence (the profiled part starts at the
    first residual_stencil_kernel launch, after the global solves that build
    the sequence).  3D cases: the
    anisotropic n^3 system from x0 = 0 (fp64_3d: one pcg_kernel launch;
    mixed3d: Alg 1 with FP32 inner CG, one ir_kernel launch).  csr3t: the 3T
    system on an n x n grid, one global pcg_kernel launch.  batched: the
    first --systems systems of the 512-system batch solved once without
    graph capture (one batched_kernel launch).  heat: the first linear
    system of the nonlinear heat test on an n x n grid, by the global PCG and
    then by Alg 1 with gradient marking."""
    import numpy as np
    import torch

    import gen
    import paper_2001_01158_gb300 as lcg

    lcg.build()
    dev = torch.device("cuda", 0)
    T = lambda v, dt=torch.float64: torch.as_tensor(v, dtype=dt, device=dev)  # noqa: E731
    ctx = lcg.Context(0)
    sp = lcg.SolveParams(1e-8, 200000, lcg.PREC_FP64, 0.0, 0)
    st = lcg.Stats()
    kind, n = args.profile_case, args.n
    if kind in ("global2d", "alg1", "alg1_rel", "alg1_gradient", "mixed2d"):
        d = gen.cfg2_fronts2d(seed=0, n=n)
        op, seq = d["op"], d["seq"]
        gop = lcg.StencilOperator(ctx, op.shape, T(op.D), T(op.Tx), T(op.Ty))
        x1 = torch.zeros(op.n, dtype=torch.float64, device=dev)
        lcg.pcg_solve(ctx, gop, T(seq.source(1)), x1, sp)
        b2 = x1 / op.meta["dt"] + T(seq.source(2))
        x = x1.clone()
        if kind == "global2d":
            lcg.pcg_solve(ctx, gop, b2, x, sp, st)
        elif kind == "mixed2d":   # the mixed-precision global solve (one ir_kernel launch)
            lcg.pcg_solve(ctx, gop, b2, x, lcg.SolveParams(1e-8, 200000, lcg.PREC_MIXED, 1e-4, 30), st)
        else:
            mark = {"alg1": MARK_ALG3, "alg1_rel": MARK_REL, "alg1_gradient": MARK_GRAD}[kind]
            lcg.solve_local_then_global(ctx, gop, b2, x, lcg.default_params(**mark, tol=1e-8), st)
    elif kind == "alg1_steps":
        d = gen.cfg2_fronts2d(seed=0, n=n)
        op, seq = d["op"], d["seq"]
        gop = lcg.StencilOperator(ctx, op.shape, T(op.D), T(op.Tx), T(op.Ty))
        k_max = min(args.systems, seq.steps)
        xs = [torch.zeros(op.n, dtype=torch.float64, device=dev)]
        for k in range(1, k_max + 1):   # the sequence's previous solutions, by the global PCG
            x = xs[-1].clone()
            lcg.pcg_solve(ctx, gop, xs[-1] / op.meta["dt"] + T(seq.source(k)), x, sp)
            xs.append(x)
        prm = lcg.default_params(**MARK_ALG3, tol=1e-8)
        for k in range(1, k_max + 1):
            x = xs[k - 1].clone()
            lcg.solve_local_then_global(ctx, gop, xs[k - 1] / op.meta["dt"] + T(seq.source(k)), x, prm, st)
    elif kind in ("fp64_3d", "mixed3d"):
        d = gen.cfg3_aniso3d(seed=0, n=n)
        op = d["op"]
        gop = lcg.StencilOperator(ctx, op.shape, T(op.D), T(op.Tx), T(op.Ty), T(op.Tz))
        x = T(d["x0"])
        if kind == "fp64_3d":
            lcg.pcg_solve(ctx, gop, T(d["b"]), x, lcg.SolveParams(1e-10, 200000, lcg.PREC_FP64, 0.0, 0), st)
        else:
            prm = lcg.default_params(lcg.MARK_RESIDUAL, lcg.THR_REL_MAX, 1e-3, lcg.EXP_DILATE, 2, tol=1e-10,
                                     precision=lcg.PREC_MIXED, inner_tol=1e-5)
            lcg.solve_local_then_global(ctx, gop, T(d["b"]), x, prm, st)
    elif kind == "heat":   # the first linear system of the heat test (Sec. 3.2) on n x n cells
        xc = (np.arange(n) + 0.5) / n
        T0 = T(np.tile(np.exp(-100.0 * xc) + 1e-4, n))
        bt, bv = [lcg.BC_DIRICHLET, lcg.BC_DIRICHLET, lcg.BC_NEUMANN, lcg.BC_NEUMANN], [1.0, 1e-4, 0.0, 0.0]
        D, Tx, Ty, b = (torch.empty(n * n, dtype=torch.float64, device=dev) for _ in range(4))
        lcg.heat2d_assemble(ctx, (n, n), 1.0 / n, 1e-2, bt, bv, T0 ** 3.5, T0, D, Tx, Ty, b)
        gop = lcg.StencilOperator(ctx, (n, n, 1), D, Tx, Ty)
        x = T0.clone()
        lcg.pcg_solve(ctx, gop, b, x, lcg.SolveParams(1e-10, 100000, lcg.PREC_FP64, 0.0, 0), st)
        x = T0.clone()
        lcg.solve_local_then_global(ctx, gop, b, x,
                                    lcg.default_params(lcg.MARK_GRADIENT, alpha=1e-4, grad_layers=0, tol=1e-10), st)
    elif kind == "csr3t":
        rp, ci, av = gen.threeT_2d(11, n, n)
        rng = np.random.default_rng(5)
        x0 = 1.0 + 0.1 * rng.standard_normal(len(rp) - 1)
        b = gen.csr_matvec(rp, ci, av, x0)
        b[3 * (n * (n // 2) + n // 2)] += 1.0
        gop = lcg.CsrOperator(ctx, T(rp, torch.int32), T(ci, torch.int32), T(av))
        x = T(x0)
        lcg.pcg_solve(ctx, gop, T(b), x, sp, st)
    else:
        items = gen.cfg4_batch(seed=0)[:args.systems]
        systems = [(it["op"].shape[0], it["op"].shape[1], T(it["op"].D), T(it["op"].Tx), T(it["op"].Ty))
                   for it in items]
        batch = lcg.Batch(ctx, systems)
        x = T(np.concatenate([it["x0"] for it in items]))
        batch.solve(T(np.concatenate([it["b"] for it in items])), x,
                    lcg.batch_params(beta=1e-3, layers=2, tol=1e-8, inner_tol=1e-4))
        torch.cuda.synchronize(dev)
        s = batch.stats()
        print(json.dumps({"case": kind, "systems": len(s), "cells": batch.cells,
                          "inner_iterations_mean": statistics.mean(v["it_global"] for v in s)}))
        return
    torch.cuda.synchronize(dev)
    print(json.dumps({"case": kind, "n": n, **st.as_dict()}))


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
    rank, ws, local = dist_init(args)
    try:
        if args.impl == "reference":
            run_reference(args, rank, ws)
        else:
            run_gpu(args, rank, ws, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
