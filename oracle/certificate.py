"""O3: Schwartz-Zippel certificate for determinants too large for O1/O2.

A claimed det(A) (dense lex coefficients over the box prod [0, D_v]) is
evaluated at random points r of F_q^k, q a 61-bit prime outside the NTT prime
range, and compared with det(A(r)) mod q by Gaussian elimination.  A wrong
claim passes one point with probability at most (sum_v D_v) / q, so ``trials``
independent points bound a false pass by that number to the power ``trials``.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import poly as P
from .modular import det_mod_p

Q61 = (1 << 61) - 1  # Mersenne prime, not of the NTT form used by the method


def _eval_dense(vec: Sequence[int], degs: Sequence[int], point: Sequence[int], q: int) -> int:
    s = 0
    for e, c in zip(P.lex_exponents(degs), vec):
        c = int(c)
        if not c:
            continue
        t = c % q
        for x, ev in zip(point, e):
            t = t * pow(x, ev, q) % q
        s += t
    return s % q


def _eval_horner(box, degs: Sequence[int], point: Sequence[int], q: int) -> int:
    """The value _eval_dense gives, by nested Horner: ``box`` holds the
    coefficients mod q as an object array shaped (d_1+1, ..., d_k+1) (lex, x_1
    slowest, so the last axis is x_k); each step folds the last axis,
    acc = acc * x_v + slice, over whole slices at once."""
    acc = box
    for v in range(len(degs) - 1, -1, -1):
        x = int(point[v])
        h = acc[..., -1]
        for e in range(int(degs[v]) - 1, -1, -1):
            h = (h * x + acc[..., e]) % q
        acc = h
    return int(acc) % q


def _box(vec: Sequence[int], degs: Sequence[int], q: int):
    arr = np.empty(len(vec), dtype=object)
    arr[:] = [int(c) for c in vec]
    return (arr % q).reshape(tuple(int(d) + 1 for d in degs))


def check(coeffs, degs: Sequence[int], claimed: Sequence[int], D: Sequence[int],
          seed: int = 12345, trials: int = 8, q: int = Q61) -> bool:
    """True when the claimed determinant agrees with det(A(r)) mod q at every
    one of ``trials`` random points (the claimed polynomial is evaluated by
    nested Horner, the entries by the plain sum over their monomials)."""
    rng = np.random.default_rng(seed)
    n = len(coeffs)
    k = len(degs)
    box = _box(claimed, D, q)
    for _ in range(trials):
        point = [int(x) for x in rng.integers(1, q - 1, k, dtype=np.int64)]
        A = [[_eval_dense(coeffs[i][j], degs, point, q) for j in range(n)] for i in range(n)]
        if det_mod_p(A, q) != _eval_horner(box, D, point, q):
            return False
    return True
