"""Autotuner for the ragged-batch kernel: times every launch configuration
(block size, tile) on the caller's batch with graph replays and keeps the
fastest, cached in a JSON file keyed by device and batch shape.

Cache file: $BOYS_AUTOTUNE_CACHE, else ~/.cache/boys_gb300/autotune.json.
"""
from __future__ import annotations

import json
import math
import os

import torch

from .api import RaggedBatch, ragged_variants


def _cache_path() -> str:
    return os.environ.get("BOYS_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "boys_gb300", "autotune.json"
    )


def _key(batch: RaggedBatch) -> str:
    name = torch.cuda.get_device_name(batch.device)
    # bucket the shape so similar batches share an entry
    r = int(math.log2(max(1, batch.num_requests)))
    a = int(math.log2(max(1, batch.x_size)))
    return f"{name}|ragged_f64|R2^{r}|args2^{a}"


def _load() -> dict:
    try:
        with open(_cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(cache: dict) -> None:
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def time_variant(batch: RaggedBatch, x: torch.Tensor, out: torch.Tensor, variant: int, reps: int = 5) -> float:
    """Median milliseconds of one graph replay of the batch with a variant."""
    g = batch.capture(x, out, variant)
    stream = torch.cuda.current_stream(batch.device)
    times = []
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    times = sorted(times[1:])
    return times[len(times) // 2]


def tune_ragged(batch: RaggedBatch, x: torch.Tensor, out: torch.Tensor | None = None, use_cache: bool = True,
                reps: int = 5) -> dict:
    """Pick the fastest variant for this batch; returns {"variant", "ms", "all"}."""
    cache = _load() if use_cache else {}
    key = _key(batch)
    if use_cache and key in cache:
        return cache[key]
    if out is None:
        out = torch.empty(batch.out_size, dtype=torch.float64, device=batch.device)
    results = []
    for v, (block, tile) in enumerate(ragged_variants()):
        ms = time_variant(batch, x, out, v, reps)
        results.append({"variant": v, "block": block, "tile": tile, "ms": round(ms, 5)})
    best = min(results, key=lambda d: d["ms"])
    entry = {"variant": best["variant"], "ms": best["ms"], "all": results}
    if use_cache:
        cache[key] = entry
        _store(cache)
    return entry
