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

from .binding import EBOUND, Plan, PolydetError, as_u32, hadamard_primes, limbs_to_ints
from .resume import ResidueStore, input_digest


@dataclass
class DetResult:
    coeffs: List[int]      # lex over the box prod [0, D_v]
    D: tuple
    P: int
    W: int
    limbs: np.ndarray      # [C][W] uint32


def entry_l1(coeffs: np.ndarray) -> np.ndarray:
    """[n][n] l1 norms of the entries' coefficient vectors."""
    return np.abs(np.asarray(coeffs, dtype=np.int64)).sum(axis=-1)


def prime_count(coeffs: np.ndarray) -> int:
    return hadamard_primes(entry_l1(coeffs))[0]


def _chunk(plan: Plan, budget_bytes: int) -> int:
    per_prime = 4 * (plan.n * plan.n * plan.G + plan.G + max(plan.eval_ws_words, plan.interp_ws_words))
    return max(1, min(plan.P, budget_bytes // max(1, per_prime)))


def determinant(coeffs: np.ndarray, degs: Sequence[int], nprimes: Optional[int] = None,
                store: Optional[ResidueStore] = None, budget_bytes: int = 8 << 30,
                stream: Optional[torch.cuda.Stream] = None,
                stop_after_chunks: Optional[int] = None, full_grid: bool = False) -> DetResult:
    """Exact det of the polynomial matrix ``coeffs`` [n][n][E] (lex encoding
    of Sec. 2) with entry degrees ``degs``; returns its coefficients."""
    coeffs = np.asarray(coeffs)
    n = coeffs.shape[0]
    if coeffs.shape[:2] != (n, n):
        raise ValueError("coeffs must be [n][n][E]")
    if np.abs(coeffs).max(initial=0) >= 2 ** 31:
        raise ValueError("coefficients must fit in int32")
    P = nprimes if nprimes is not None else prime_count(coeffs)
    plan = Plan(n, degs, P, full_grid=full_grid)
    dev = torch.device("cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(st):
        c_dev = torch.from_numpy(np.ascontiguousarray(coeffs, dtype=np.int32).reshape(-1)).to(dev)
        residues = torch.empty(P * plan.C, dtype=torch.int32, device=dev)
        todo = list(range(P))
        if store is not None:
            store.open_job({"n": n, "degs": [int(d) for d in degs], "primes": plan.primes,
                            "full_grid": bool(full_grid), "input": input_digest(coeffs, degs)})
            for q, r in store.done(P, plan.C).items():
                residues[q * plan.C:(q + 1) * plan.C].copy_(torch.from_numpy(r.view(np.int32)))
                todo.remove(q)
        ch = _chunk(plan, budget_bytes)
        evals = torch.empty(ch * n * n * plan.G, dtype=torch.int32, device=dev) if todo else None
        detv = torch.empty(ch * plan.G, dtype=torch.int32, device=dev) if todo else None
        ws = plan.workspace(ch) if todo else None
        runs: List[List[int]] = []  # consecutive primes, at most ch per launch
        for q in todo:
            if runs and runs[-1][1] == q and runs[-1][1] - runs[-1][0] < ch:
                runs[-1][1] = q + 1
            else:
                runs.append([q, q + 1])
        for done, (lo, hi) in enumerate(runs):
            if stop_after_chunks is not None and done >= stop_after_chunks:
                raise InterruptedError("stopped after the requested number of chunks")
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
        limbs = torch.empty(plan.C * plan.W, dtype=torch.int32, device=dev)
        plan.crt(residues, limbs, st)
        status = plan.sync_status(st)
        if status:
            raise PolydetError(EBOUND, f"device status {status:#x}")
        host_limbs = as_u32(limbs).reshape(plan.C, plan.W)
    out = DetResult(limbs_to_ints(host_limbs, plan.W), plan.D, plan.P, plan.W, host_limbs)
    plan.close()
    return out
