"""Autotuner for the fused kernels' launch shape.

For every matrix order present in a batch it times the fused kernel of that
order alone (CUDA events on the launching stream, after one untimed launch)
for each admissible CTA size, keeps the fastest, and records the choice in a
JSON cache keyed by device name, matrix order and a bucket of the work size,
so later batches on the same device skip the search.  The choice only moves
work between CTAs: results are identical for every candidate.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Optional

import torch

CACHE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune")
CACHE = os.path.join(CACHE_DIR, "fused_launch.json")


def team(n: int) -> int:
    return 1 if n <= 14 else (2 if n <= 18 else (4 if n <= 28 else 8))


def candidates(n: int):
    return [t for t in (32, 64, 128) if t % team(n) == 0]


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d: dict) -> None:
    os.makedirs(CACHE_DIR, exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _key(n: int, items: int) -> str:
    dev = torch.cuda.get_device_name().replace(" ", "_")
    return f"{dev}/n{n}/items2^{int(math.log2(max(1, items)))}"


def apply_cached(batch) -> Dict[int, dict]:
    """Set every order that has a cached choice; leave the others alone."""
    cache = _load()
    out = {}
    for n in batch.orders():
        key = _key(n, int(batch.info.items[n]))
        if key in cache:
            batch.set_launch(n, cache[key]["threads"])
            out[n] = dict(cache[key], cached=True)
    return out


def tune(batch, partial, detvals, ws, stream: Optional[torch.cuda.Stream] = None,
         reps: int = 2, use_cache: bool = True) -> Dict[int, dict]:
    """Pick the CTA size of every order in ``batch`` (a binding.Batch whose
    partial tensor has been computed); returns {n: {threads, ms}}."""
    st = stream or torch.cuda.current_stream()
    cache = _load() if use_cache else {}
    chosen = {}
    for n in batch.orders():
        key = _key(n, int(batch.info.items[n]))
        if use_cache and key in cache:
            batch.set_launch(n, cache[key]["threads"])
            chosen[n] = dict(cache[key], cached=True)
            continue
        best = None
        timings = {}
        for th in candidates(n):
            batch.set_launch(n, th)
            batch.condense(partial, detvals, ws, st, n=n)  # untimed
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(st)
            for _ in range(reps):
                batch.condense(partial, detvals, ws, st, n=n)
            e.record(st)
            e.synchronize()
            ms = s.elapsed_time(e) / reps
            timings[th] = ms
            if best is None or ms < best[1]:
                best = (th, ms)
        batch.set_launch(n, best[0])
        chosen[n] = {"threads": best[0], "ms": best[1], "tried": timings}
        cache[key] = {"threads": best[0], "ms": best[1]}
    if use_cache:
        _save(cache)
    return chosen
