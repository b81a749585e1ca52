"""The plain (one matrix at a time) determinant: Algorithm 1 of the paper.

For every prime: evaluation (polydet_eval), condensation
(polydet_condense_batch), interpolation (polydet_interp); then mixed-radix
CRT over all primes (polydet_crt).  Primes are processed in chunks sized to a
device-memory budget; with a ``ResidueStore`` the per-prime residues are
saved after each chunk, once the device status word reads clean, and a
rerun computes only the missing primes.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from .binding import (EBOUND, Plan, PolydetError, as_u32, det_degree_bound, entry_degrees,
                      hadamard_primes, limbs_to_ints)
from .binding import unique_entries as unique_entries_of
from .resume import ResidueStore, input_digest


@dataclass
class DetResult:
    coeffs: Optional[List[int]]  # lex over the box prod [0, D_v] (None: as_ints=False)
    D: tuple
    P: int
    W: int
    limbs: np.ndarray      # [C][W] uint32
    primes_bound: int = -1  # primes of the coefficient bound (P is fewer after an early stop)


def unpermute_output(vals: Sequence[int], order: Sequence[int], box: Sequence[int]) -> List[int]:
    """Output coefficients computed with the variables in ``order`` (lex over
    ``box``, the extents D_v + 1 in that order) put back in the caller's
    variable order: the inverse of the transposition ``permute_coeffs``
    applies to the input."""
    if list(order) == sorted(order):
        return list(vals)
    arr = np.empty(len(vals), dtype=object)
    arr[:] = list(vals)
    inv = [list(order).index(v) for v in range(len(order))]
    return arr.reshape(tuple(int(b) for b in box)).transpose(inv).reshape(-1).tolist()


def permute_coeffs(coeffs: np.ndarray, degs: Sequence[int], order: Sequence[int]) -> np.ndarray:
    """[n][n][E] lex coefficients with the variables taken in ``order``."""
    n = coeffs.shape[0]
    t = np.asarray(coeffs).reshape((n, n) + tuple(int(d) + 1 for d in degs))
    return t.transpose((0, 1) + tuple(2 + v for v in order)).reshape(n, n, -1)


def entry_l1(coeffs: np.ndarray) -> np.ndarray:
    """[n][n] l1 norms of the entries' coefficient vectors."""
    return np.abs(np.asarray(coeffs, dtype=np.int64)).sum(axis=-1)


def prime_count(coeffs: np.ndarray) -> int:
    return hadamard_primes(entry_l1(coeffs))[0]


def _chunk(plan: Plan, budget_bytes: int) -> int:
    per_prime = 4 * (plan.entries * plan.G + plan.G + max(plan.eval_ws_words, plan.interp_ws_words))
    return max(1, min(plan.P, budget_bytes // max(1, per_prime)))


def determinant(coeffs: np.ndarray, degs: Sequence[int], nprimes: Optional[int] = None,
                store: Optional[ResidueStore] = None, budget_bytes: int = 8 << 30,
                stream: Optional[torch.cuda.Stream] = None,
                stop_after_chunks: Optional[int] = None, full_grid: bool = False,
                tight_degrees: bool = False, unique_entries: bool = False,
                streamed: Optional[bool] = None, as_ints: bool = True,
                early_stop: bool = False) -> DetResult:
    """Exact det of the polynomial matrix ``coeffs`` [n][n][E] (lex encoding
    of Sec. 2) with entry degrees ``degs``; returns its coefficients over the
    box prod [0, D_v].

    ``tight_degrees``: D_v from the entries' degrees (the assignment bound of
    polydet_det_degree_bound) instead of n d_v.  ``unique_entries``: evaluate
    each distinct entry once (polydet_plan_set_entry_map).  ``streamed``:
    evaluation and condensation slab by slab through a workspace within
    ``budget_bytes`` (polydet_eval_condense), one prime at a time, with the
    variable of lowest degree taken first (its nodes are the slabs); None
    streams exactly when one prime's evaluated matrices exceed the budget.
    ``as_ints``: False leaves ``coeffs`` None (outputs of hundreds of
    millions of coefficients are read from ``limbs``).  ``early_stop``:
    primes one at a time, and stop at the first prime that leaves every
    coefficient's reconstruction unchanged (polydet_crt_check); P is then
    the primes used, ``primes_bound`` the count of the coefficient bound."""
    coeffs = np.asarray(coeffs)
    n = coeffs.shape[0]
    if coeffs.shape[:2] != (n, n):
        raise ValueError("coeffs must be [n][n][E]")
    if np.abs(coeffs).max(initial=0) >= 2 ** 31:
        raise ValueError("coefficients must fit in int32")
    degs = tuple(int(d) for d in degs)
    P = nprimes if nprimes is not None else prime_count(coeffs)
    order = list(range(len(degs)))
    if streamed is not False:
        order = sorted(order, key=lambda v: (degs[v], v))
    cp = permute_coeffs(coeffs, degs, order)
    dp = tuple(degs[v] for v in order)
    D = None
    if tight_degrees:
        D = det_degree_bound(entry_degrees(cp, dp), len(dp))
    plan = Plan(n, dp, P, full_grid=full_grid, det_degs=D)
    rows = np.ascontiguousarray(cp, dtype=np.int32).reshape(n * n, -1)
    if unique_entries:
        emap, U, uniq = unique_entries_of(cp)
        plan.set_entry_map(emap, U)
        rows = uniq
    if streamed is None:
        streamed = 4 * (plan.entries * plan.G + plan.G) > budget_bytes
    if not streamed and order != sorted(order):  # the plain path keeps the caller's order
        plan.close()
        return determinant(coeffs, degs, nprimes=P, store=store, budget_bytes=budget_bytes,
                           stream=stream, stop_after_chunks=stop_after_chunks, full_grid=full_grid,
                           tight_degrees=tight_degrees, unique_entries=unique_entries, streamed=False,
                           as_ints=as_ints, early_stop=early_stop)
    dev = torch.device("cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(st):
        flat = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1)
        c_dev = torch.from_numpy(flat if flat.size else np.zeros(1, dtype=np.int32)).to(dev)
        residues = torch.empty(P * plan.C, dtype=torch.int32, device=dev)
        todo = list(range(P))
        if store is not None:
            store.open_job({"n": n, "degs": [int(d) for d in degs], "primes": plan.primes,
                            "full_grid": bool(full_grid), "input": input_digest(coeffs, degs),
                            "det_degs": [int(x) for x in plan.D], "order": order})
            for q, r in store.done(P, plan.C).items():
                residues[q * plan.C:(q + 1) * plan.C].copy_(torch.from_numpy(r.view(np.int32)))
                todo.remove(q)
        if early_stop and store is not None:
            raise ValueError("early_stop and a residue store do not combine")
        if streamed:
            ch = 1
            ws_words = max(plan.stream_ws_words(1), plan.interp_ws_words,
                           min(plan.stream_ws_words(plan.M[0]), max(0, budget_bytes // 4 - plan.G)))
            evals = None
            ws = torch.empty(ws_words, dtype=torch.int32, device=dev) if todo else None
        else:
            ch = 1 if early_stop else _chunk(plan, budget_bytes)
            evals = torch.empty(ch * plan.entries * plan.G, dtype=torch.int32, device=dev) if todo else None
            ws = plan.workspace(ch) if todo else None
        detv = torch.empty(ch * plan.G, dtype=torch.int32, device=dev) if todo else None
        runs: List[List[int]] = []  # consecutive primes, at most ch per launch
        for q in todo:
            if runs and runs[-1][1] == q and runs[-1][1] - runs[-1][0] < ch:
                runs[-1][1] = q + 1
            else:
                runs.append([q, q + 1])
        used = P
        if early_stop:
            digits = torch.empty(P * plan.C, dtype=torch.int32, device=dev)
            unstable = torch.zeros(1, dtype=torch.int32, device=dev)
        for done, (lo, hi) in enumerate(runs):
            if stop_after_chunks is not None and done >= stop_after_chunks:
                raise InterruptedError("stopped after the requested number of chunks")
            if streamed:
                plan.eval_condense(c_dev, lo, hi, detv, ws, st)
            else:
                plan.eval(c_dev, lo, hi, evals, ws, st)
                plan.condense(evals, lo, hi, detv, st)
            plan.interp(detv, lo, hi, residues[lo * plan.C:hi * plan.C], ws, st)
            if store is not None:
                # a restart point is only as good as its residues: read the
                # status word first, and persist nothing the device flagged
                status = plan.sync_status(st)
                if status:
                    raise PolydetError(EBOUND, f"device status {status:#x} in primes [{lo}, {hi}); "
                                               "nothing saved for them")
                host = as_u32(residues[lo * plan.C:hi * plan.C])
                for q in range(lo, hi):
                    store.save(q, host[(q - lo) * plan.C:(q - lo + 1) * plan.C])
            if early_stop and lo >= 1:
                plan.crt_check(residues, digits, lo, unstable, st)
                if int(unstable.item()) == 0:  # prime lo changed no coefficient: stop
                    used = lo + 1
                    break
                unstable.zero_()
        del evals, ws, detv
        cplan = plan if used == P else Plan(n, dp, used, full_grid=full_grid, det_degs=D)
        limbs = torch.empty(cplan.C * cplan.W, dtype=torch.int32, device=dev)
        cplan.crt(residues, limbs, st)
        status = plan.sync_status(st)
        if status:
            raise PolydetError(EBOUND, f"device status {status:#x}")
        host_limbs = as_u32(limbs).reshape(cplan.C, cplan.W)
        W = cplan.W
        if cplan is not plan:
            cplan.close()
    box = tuple(int(x) + 1 for x in plan.D)
    vals = limbs_to_ints(host_limbs, W) if as_ints else None
    Dc = [0] * len(degs)
    for i, v in enumerate(order):
        Dc[v] = plan.D[i]
    if order != sorted(order):
        if as_ints:
            vals = unpermute_output(vals, order, box)
        inv = [order.index(v) for v in range(len(order))]
        host_limbs = host_limbs.reshape(box + (W,)).transpose(tuple(inv) + (len(order),)).reshape(-1, W)
    out = DetResult(vals, tuple(Dc), used, W, np.ascontiguousarray(host_limbs), primes_bound=P)
    plan.close()
    return out
