"""Host-side planning quantities of Sec. 2: degree bounds, grid sizes, the
coefficient bound ("boundary") and the number of primes.

Readings of the paper used here (the paper states no formula for either):

* Degree bound.  det(A) has degree at most sum_i max_j deg_v a_ij <= n * d_v in
  x_v, where d_v bounds the degree of every entry in x_v; the assignment
  bound (the largest sum_i deg_v a_{i s(i)} over permutations s) is tighter
  still and is what structured inputs (Sylvester matrices) are planned with.  The grid needs
  D_v + 1 distinct nodes per variable (interpolation, Sec. 3.3), padded to the
  next power of two, N_v = nextpow2(D_v + 1), which reproduces the paper's
  example (15, 7, 9) -> (16, 8, 16) of Sec. 2.
* Coefficient bound.  A coefficient of det(A) is a Fourier coefficient of
  z -> det A(z) on the unit torus, so it is at most max |det A(z)| there; by
  Hadamard's inequality and |a_ij(z)| <= ||a_ij||_1 that is at most
  prod_i (sum_j ||a_ij||_1^2)^(1/2) (rows; the column form also holds and the
  smaller is used).  Signs are recovered by the symmetric lift, so the primes
  must satisfy prod p > 2 * bound (Sec. 2 asks only prod p >= bound).
"""
from __future__ import annotations

from math import prod
from typing import List, Sequence, Tuple


def next_pow2(x: int) -> int:
    n = 1
    while n < x:
        n *= 2
    return n


def det_degree_bound(n: int, degs: Sequence[int]) -> Tuple[int, ...]:
    """D_v = n * d_v: the degree bound of det(A) in each variable."""
    return tuple(n * int(d) for d in degs)


def entry_degrees(coeffs, degs: Sequence[int]):
    """Per entry of the dense lex matrix ``coeffs`` [n][n][E]: its degree in
    each variable, or None for an identically zero entry."""
    from itertools import product
    exps = list(product(*[range(int(d) + 1) for d in degs]))
    out = []
    for row in coeffs:
        r = []
        for vec in row:
            nz = [e for e, c in zip(exps, vec) if int(c) != 0]
            r.append(None if not nz else tuple(max(e[v] for e in nz) for v in range(len(degs))))
        out.append(r)
    return out


def assignment_degree_bound(edeg, k: int, brute: "bool | None" = None) -> Tuple[int, ...]:
    """D_v = max over permutations s with every a_{i s(i)} nonzero of
    sum_i deg_v a_{i s(i)}: each term of the Leibniz expansion of det(A) is
    such a product, so deg_v det(A) <= D_v (0 when no permutation avoids the
    zero entries: then det(A) = 0).  It never exceeds the row-sum bound
    sum_i max_j deg_v a_ij nor the column-sum bound.  Brute force over all
    permutations for n <= 7 (or when ``brute``), otherwise the maximum-weight
    perfect matching of scipy's assignment solver, zero entries weighted
    below any matching that avoids them."""
    from itertools import permutations
    n = len(edeg)
    out = []
    for v in range(k):
        if (n <= 7) if brute is None else brute:
            best = None
            for s in permutations(range(n)):
                if any(edeg[i][s[i]] is None for i in range(n)):
                    continue
                t = sum(edeg[i][s[i]][v] for i in range(n))
                best = t if best is None or t > best else best
            out.append(0 if best is None else best)
        else:
            import numpy as np
            from scipy.optimize import linear_sum_assignment
            big = 1 + sum(max((e[v] for e in r if e is not None), default=0) for r in edeg)
            w = np.array([[(e[v] if e is not None else -big * (n + 1)) for e in r] for r in edeg],
                         dtype=np.int64)
            rows, cols = linear_sum_assignment(w, maximize=True)
            if any(edeg[i][j] is None for i, j in zip(rows, cols)):
                out.append(0)
            else:
                out.append(int(w[rows, cols].sum()))
    return tuple(out)


def grid_sizes(D: Sequence[int]) -> Tuple[int, ...]:
    """N_v = nextpow2(D_v + 1) evaluation nodes per variable."""
    return tuple(next_pow2(int(d) + 1) for d in D)


def paper_padding(degs: Sequence[int]) -> Tuple[Tuple[int, ...], int]:
    """Sec. 2: degree vector -> padded power-of-two sizes and q_max."""
    Ns = grid_sizes(degs)
    qmax = max(N.bit_length() - 1 for N in Ns)
    return Ns, qmax


def entry_l1(coeffs, n: int) -> List[List[int]]:
    return [[sum(abs(int(c)) for c in coeffs[i][j]) for j in range(n)] for i in range(n)]


def hadamard_bound_sq(coeffs, degs: Sequence[int]) -> int:
    """Square of the coefficient bound: min over rows/columns of
    prod_i sum_j ||a_ij||_1^2, as an exact integer."""
    n = len(coeffs)
    l1 = entry_l1(coeffs, n)
    rows = prod(sum(l1[i][j] ** 2 for j in range(n)) for i in range(n))
    cols = prod(sum(l1[i][j] ** 2 for i in range(n)) for j in range(n))
    return min(rows, cols)


MIN_PRIMES = 2  # Sec. 4.1: never fewer than two large primes


def primes_needed(bound_sq: int, primes: Sequence[int], min_primes: int = MIN_PRIMES) -> int:
    """Smallest P >= min_primes with prod_{i<P} p_i > 2 * bound, i.e.
    (prod p)^2 > 4 * bound^2."""
    m = 1
    for i, p in enumerate(primes):
        m *= p
        if i + 1 >= min_primes and m * m > 4 * bound_sq:
            return i + 1
    raise ValueError("prime table too short for this bound")


def output_words(primes: Sequence[int]) -> int:
    """W: 32-bit words of the two's-complement output; (-M/2, M/2) fits in
    32*W bits when M = prod p < 2^(32 W)."""
    M = prod(primes)
    return max(1, (M.bit_length() + 31) // 32)
