"""Autotuner for the batched launch: picks the CTA size and the number of
CTAs per SM by timing CUDA-graph replays of the batch's own solve, and
caches the choice in a JSON file keyed by the GPU and the batch's size class.

    from paper_2001_01158_gb300.autotune import tune_batch
    cfg = tune_batch(batch, b, x0, params)      # applies the best config

The cache file defaults to ~/.cache/lc_autotune.json (LC_AUTOTUNE_CACHE
overrides it).  A cached choice is applied without timing.
"""
from __future__ import annotations

import json
import math
import os

import torch

BLOCKS = (256, 512, 1024)
CTAS_PER_SM = (0, 1, 2)


def _cache_path() -> str:
    return os.environ.get("LC_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "lc_autotune.json"))


def size_class(batch) -> str:
    """Coarse description of a batch: count and log2 of the mean and max system size."""
    mean = batch.cells / max(1, batch.nsys)
    return f"n{batch.nsys}-mean2^{round(math.log2(max(1.0, mean)))}-max2^{round(math.log2(max(batch.sizes)))}"


def _key(batch) -> str:
    return f"{torch.cuda.get_device_name()}|batched|{size_class(batch)}"


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


def time_config(batch, b, x0, params, block, ctas, reps=2) -> float:
    """Milliseconds of one graph replay (min of `reps`) for a configuration."""
    batch.set_tuning("block", block)
    batch.set_tuning("ctas_per_sm", ctas)
    x = x0.clone()
    batch.capture(b, x, params)
    best = float("inf")
    for _ in range(reps + 1):
        x.copy_(x0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.replay()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_batch(batch, b, x0, params, use_cache=True, verbose=False) -> dict:
    """Choose and apply the fastest (block, ctas_per_sm); returns the choice."""
    key = _key(batch)
    cache = load_cache() if use_cache else {}
    if key in cache:
        cfg = cache[key]
    else:
        results = []
        for block in BLOCKS:
            for ctas in CTAS_PER_SM:
                ms = time_config(batch, b, x0, params, block, ctas)
                results.append((ms, block, ctas))
                if verbose:
                    print(f"autotune {key}: block={block} ctas_per_sm={ctas}: {ms:.3f} ms", flush=True)
        ms, block, ctas = min(results)
        cfg = {"block": block, "ctas_per_sm": ctas, "ms": ms, "candidates": [list(r) for r in results]}
        if use_cache:
            cache[key] = cfg
            _save_cache(cache)
    batch.set_tuning("block", cfg["block"])
    batch.set_tuning("ctas_per_sm", cfg["ctas_per_sm"])
    return cfg
