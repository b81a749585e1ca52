"""O3: Schwartz-Zippel certificate for determinants too large for O1/O2
(``check`` on Python integers; ``check_limbs`` on the limbs of outputs too
large for them).

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


# ---------------------------------------------------------------------------
# The same certificate for outputs too large for Python integers (hundreds
# of millions of coefficients): the claimed coefficients are taken straight
# from their two's-complement 32-bit limbs and reduced mod q = 2^31 - 1 (a
# Mersenne prime; q - 1 = 2 (2^30 - 1), so it is not of the NTT form c 2^20 + 1),
# small enough that every product of two residues fits in 64 bits.  A wrong
# claim passes one point with probability at most (sum_v D_v) / q.
# ---------------------------------------------------------------------------
Q31 = (1 << 31) - 1


def limbs_mod_q(limbs: np.ndarray, q: int = Q31) -> np.ndarray:
    """[C][W] little-endian two's-complement uint32 words -> each value mod q
    (int64 in [0, q)), by Horner over the words from the top one down."""
    L = np.ascontiguousarray(limbs, dtype=np.uint32)
    C, W = L.shape
    base = (1 << 32) % q
    acc = np.zeros(C, dtype=np.int64)
    for w in range(W - 1, -1, -1):
        acc = (acc * base + L[:, w].astype(np.int64)) % q
    neg = (L[:, W - 1] >> 31).astype(bool)  # the value is U - 2^(32 W)
    acc[neg] = (acc[neg] - pow(2, 32 * W, q)) % q
    return acc


def _horner_u64(vals: np.ndarray, point: Sequence[int], q: int) -> np.ndarray:
    """Evaluate the trailing len(point) axes of ``vals`` (residues mod q,
    int64) at ``point``: nested Horner from the last axis inwards."""
    acc = vals
    for x in reversed([int(v) % q for v in point]):
        h = acc[..., -1].copy()
        for e in range(acc.shape[-1] - 2, -1, -1):
            h = (h * x + acc[..., e]) % q
        acc = h
    return acc


def check_limbs(coeffs, degs: Sequence[int], limbs: np.ndarray, D: Sequence[int],
                seed: int = 12345, trials: int = 8, q: int = Q31) -> bool:
    """True when the determinant claimed as limbs [C][W] (lex over the box
    prod [0, D_v]) agrees with det(A(r)) mod q at every one of ``trials``
    random points r."""
    rng = np.random.default_rng(seed)
    c = np.asarray(coeffs, dtype=np.int64)
    n = c.shape[0]
    A_all = (c % q).reshape((n, n) + tuple(int(d) + 1 for d in degs))
    claim = limbs_mod_q(limbs, q).reshape(tuple(int(d) + 1 for d in D))
    for _ in range(trials):
        point = [int(x) for x in rng.integers(1, q - 1, len(degs), dtype=np.int64)]
        A = _horner_u64(A_all, point, q)
        if det_mod_p([[int(A[i, j]) for j in range(n)] for i in range(n)], q) != int(_horner_u64(claim, point, q)):
            return False
    return True
