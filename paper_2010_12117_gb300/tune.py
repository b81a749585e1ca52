"""Autotuner for the batched form's two knobs per matrix order.

For every matrix order present in a batch it times, on the launching stream
with CUDA events after one untimed run, stage 1 + stage 2 of that order
alone in each admissible configuration:

- mode: fused (last-variable evaluation inside the persistent determinant
  kernel) or materialized (first variable's NTT pass into the workspace,
  then the condensation kernel over it);
- CTA size of the fused kernel (32, 64 or 128 threads, a multiple of the
  lanes per determinant).

It keeps the fastest and records the choice in a JSON cache keyed by device
name, matrix order and a bucket of the work size, so later batches on the
same device skip the search.  The choice only moves work between kernels and
CTAs: results are identical for every candidate.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, Optional

import torch

from .binding import BATCH_FUSED, BATCH_MATERIALIZED, team_size

CACHE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune")
CACHE = os.path.join(CACHE_DIR, "batch_launch.json")


def team(n: int) -> int:
    return team_size(n)


def candidates(n: int):
    """(mode, threads) pairs tried for order n."""
    out = [(BATCH_FUSED, t) for t in (32, 64, 128) if t % team(n) == 0]
    return out + [(BATCH_MATERIALIZED, 128)]


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


def _apply(batch, n: int, choice: dict) -> None:
    batch.set_mode(n, choice["mode"])
    batch.set_launch(n, choice["threads"])


def apply_cached(batch) -> Dict[int, dict]:
    """Set every order that has a cached choice; leave the others alone.
    (The caller reruns stage 1 afterwards: a mode change alters it.)"""
    cache = _load()
    out = {}
    for n in batch.orders():
        key = _key(n, int(batch.info.items[n]))
        if key in cache:
            _apply(batch, n, cache[key])
            out[n] = dict(cache[key], cached=True)
    return out


def tune(batch, coeffs, partial, detvals, workspace: Callable[[int], torch.Tensor],
         stream: Optional[torch.cuda.Stream] = None, reps: int = 2,
         use_cache: bool = True) -> Dict[int, dict]:
    """Pick mode and CTA size of every order in ``batch`` (a binding.Batch
    whose coefficients are on the device); ``workspace(words)`` returns a
    device buffer of at least that many words.  Leaves stage 1 computed for
    the chosen modes; returns {n: {mode, threads, ms}}."""
    st = stream or torch.cuda.current_stream()
    cache = _load() if use_cache else {}
    chosen = {}
    for n in batch.orders():
        key = _key(n, int(batch.info.items[n]))
        if use_cache and key in cache:
            _apply(batch, n, cache[key])
            batch.eval(coeffs, partial, workspace(batch.words["workspace"]), st, n=n)
            chosen[n] = dict(cache[key], cached=True)
            continue
        best = None
        timings = {}
        for mode, th in candidates(n):
            _apply(batch, n, {"mode": mode, "threads": th})
            ws = workspace(batch.words["workspace"])

            def run():
                batch.eval(coeffs, partial, ws, st, n=n)
                batch.condense(partial, detvals, ws, st, n=n)
            run()  # untimed
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(st)
            for _ in range(reps):
                run()
            e.record(st)
            e.synchronize()
            ms = s.elapsed_time(e) / reps
            timings[f"{'materialized' if mode else 'fused'}/{th}"] = ms
            if best is None or ms < best[2]:
                best = (mode, th, ms)
        choice = {"mode": best[0], "threads": best[1], "ms": best[2]}
        _apply(batch, n, choice)
        batch.eval(coeffs, partial, workspace(batch.words["workspace"]), st, n=n)
        chosen[n] = dict(choice, tried=timings)
        cache[key] = choice
    if use_cache:
        _save(cache)
    return chosen
