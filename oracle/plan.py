"""Host-side planning quantities of Sec. 2: degree bounds, grid sizes, the
coefficient bound ("boundary") and the number of primes.

Readings of the paper used here (the paper states no formula for either):

* Degree bound.  det(A) has degree at most sum_i max_j deg_v a_ij <= n * d_v in
  x_v, where d_v bounds the degree of every entry in x_v.  The grid needs
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


MIN_PRIMES = 2  # Sec. 4.1: the method always uses at least two big primes


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
