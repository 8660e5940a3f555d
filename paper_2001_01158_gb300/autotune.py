"""Autotuner for the batched launch: picks the CTA size, whether the large
systems run on thread-block clusters (and of how many CTAs), and the size
from which a system counts as large, by timing CUDA-graph replays of the
batch's own solve; caches the choice in a JSON file keyed by the GPU and the
batch's size class.

    from paper_2001_01158_gb300.autotune import tune_batch
    cfg = tune_batch(batch, b, x0, params)      # applies the best config

Each candidate is timed as the median of several replays.  Among the
candidates within `slack` (3 %) of the fastest, the first in CANDIDATES
order wins, so that timing noise between runs does not flip the choice
between near-equal configurations.  The cache file defaults to
~/.cache/lc_autotune.json (LC_AUTOTUNE_CACHE overrides it).  A cached choice
is applied without timing.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import torch

# (block, ctas_per_sm, cluster, big_cells), in order of preference
CANDIDATES = [(1024, 0, 1, 65536), (512, 0, 1, 65536)] + \
             [(1024, 0, c, t) for c in (4, 8, 2) for t in (65536, 32768, 131072)] + \
             [(512, 0, 4, 65536), (512, 0, 8, 65536)]
KEYS = ("block", "ctas_per_sm", "cluster", "big_cells")


def _cache_path() -> str:
    return os.environ.get("LC_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "lc_autotune.json"))


def size_class(batch) -> str:
    """Coarse description of a batch: count and log2 of the mean and max system size."""
    mean = batch.cells / max(1, batch.nsys)
    return f"n{batch.nsys}-mean2^{round(math.log2(max(1.0, mean)))}-max2^{round(math.log2(max(batch.sizes)))}"


def _key(batch) -> str:
    return f"{torch.cuda.get_device_name()}|batched-v2|{size_class(batch)}"


def load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(cache: dict):
    p = _cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def apply(batch, cfg):
    for k in KEYS:
        batch.set_tuning(k, int(cfg[k]))


def time_config(batch, b, x0, params, cand, reps=5) -> float:
    """Median milliseconds of `reps` graph replays for a candidate."""
    apply(batch, dict(zip(KEYS, cand)))
    x = x0.clone()
    batch.capture(b, x, params)
    x.copy_(x0)
    batch.replay()   # warm-up
    ts = []
    for _ in range(reps):
        x.copy_(x0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune_batch(batch, b, x0, params, use_cache=True, verbose=False, slack=0.03) -> dict:
    """Choose and apply the fastest configuration; returns the choice."""
    key = _key(batch)
    cache = load_cache() if use_cache else {}
    if key in cache:
        cfg = cache[key]
    else:
        results = []
        for cand in CANDIDATES:
            ms = time_config(batch, b, x0, params, cand)
            results.append((ms,) + cand)
            if verbose:
                print(f"autotune {key}: {dict(zip(KEYS, cand))}: {ms:.3f} ms", flush=True)
        best = min(r[0] for r in results)
        pick = next(r for r in results if r[0] <= best * (1.0 + slack))
        cfg = dict(zip(KEYS, pick[1:]))
        cfg.update({"ms": pick[0], "best_ms": best, "candidates": [list(r) for r in results]})
        if use_cache:
            cache[key] = cfg
            _save_cache(cache)
    apply(batch, cfg)
    return cfg
