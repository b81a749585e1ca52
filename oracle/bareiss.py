"""The determinant over Z[x1..xk], exactly, by its plain definition.

The paper's method reaches det(A) in Z[x1..xk] exactly (Sec. 1-2: the modular
method "does not lose accuracy").  The oracle therefore computes that
determinant directly, with no modular arithmetic at all:

* ``det_bareiss_poly`` (O1): fraction-free Bareiss elimination over
  Z[x1..xk] on dict polynomials.  Every division is exact in Z[x1..xk].
* ``det_packed`` (O2): the same elimination over Z after the Kronecker
  substitution x_v -> 2^(b * stride_v).  The substitution is a ring
  homomorphism, so it commutes with the determinant, and it is invertible on
  polynomials whose degree in x_v is at most D_v and whose coefficients are
  below 2^(b-1) in magnitude (balanced base-2^b digits).  One polynomial
  product becomes one big-integer product, which makes the 12x12 trivariate
  workload reachable in Python.
* ``det_leibniz_poly``: the permutation expansion, for n <= 5 (a route that
  shares nothing with elimination).
* ``det_bareiss``: O1 for a matrix given entry by entry (dicts or dense
  coefficient arrays), returning the dense coefficient array of the result.
"""
from __future__ import annotations

from itertools import permutations
from math import prod
from typing import List, Sequence

from . import poly as P
from .plan import det_degree_bound, hadamard_bound_sq


def det_bareiss_poly(M: List[List[P.Poly]], k: int) -> P.Poly:
    """O1: fraction-free Bareiss over Z[x1..xk].

    After step c every entry (i, j) with i, j > c equals a (c+2)-minor of the
    (row-permuted) input, so dividing by the previous pivot - itself a
    leading minor - is exact.  A zero pivot is replaced by the first row below
    with a nonzero entry in that column (the sign flips); if there is none the
    determinant is zero.
    """
    A = [list(row) for row in M]
    n = len(A)
    if n == 0:
        return P.const(1, k)
    sign = 1
    prev = P.const(1, k)
    for c in range(n - 1):
        if not A[c][c]:
            r = next((i for i in range(c + 1, n) if A[i][c]), None)
            if r is None:
                return P.zero()
            A[c], A[r] = A[r], A[c]
            sign = -sign
        for i in range(c + 1, n):
            for j in range(c + 1, n):
                num = P.sub(P.mul(A[c][c], A[i][j]), P.mul(A[i][c], A[c][j]))
                A[i][j] = P.divexact(num, prev)
            A[i][c] = P.zero()
        prev = A[c][c]
    return P.scale(A[n - 1][n - 1], sign)


def det_bareiss_int(M: List[List[int]]) -> int:
    """Fraction-free Bareiss over Z (same loop as O1, on Python ints)."""
    A = [list(row) for row in M]
    n = len(A)
    if n == 0:
        return 1
    sign = 1
    prev = 1
    for c in range(n - 1):
        if A[c][c] == 0:
            r = next((i for i in range(c + 1, n) if A[i][c] != 0), None)
            if r is None:
                return 0
            A[c], A[r] = A[r], A[c]
            sign = -sign
        pc = A[c][c]
        rowc = A[c]
        for i in range(c + 1, n):
            rowi = A[i]
            aic = rowi[c]
            for j in range(c + 1, n):
                q, rem = divmod(pc * rowi[j] - aic * rowc[j], prev)
                if rem:
                    raise ArithmeticError("Bareiss division is not exact")
                rowi[j] = q
            rowi[c] = 0
        prev = pc
    return sign * A[n - 1][n - 1]


def det_leibniz_poly(M: List[List[P.Poly]], k: int) -> P.Poly:
    """sum over permutations s of sgn(s) * prod_i M[i][s(i)]; n <= 5 only."""
    n = len(M)
    if n > 6:
        raise ValueError("Leibniz expansion is for tiny matrices only")
    total = P.zero()
    for s in permutations(range(n)):
        inv = sum(1 for a in range(n) for b in range(a + 1, n) if s[a] > s[b])
        term = P.const(-1 if inv % 2 else 1, k)
        for i in range(n):
            term = P.mul(term, M[i][s[i]])
            if not term:
                break
        total = P.add(total, term)
    return total


# ---------------------------------------------------------------------------
# O2: Kronecker packing into one integer per entry.
# ---------------------------------------------------------------------------

def _strides(D: Sequence[int]) -> List[int]:
    """Mixed-radix place values of the box prod [0, D_v], x_k fastest."""
    st = [1] * len(D)
    for v in range(len(D) - 2, -1, -1):
        st[v] = st[v + 1] * (D[v + 1] + 1)
    return st


def pack(vec: Sequence[int], degs: Sequence[int], D: Sequence[int], b: int) -> int:
    """Entry (lex vector over the box prod [0, d_v]) evaluated at
    x_v = 2^(b * stride_v), where strides are those of the box prod [0, D_v]."""
    assert b % 8 == 0
    nb = b // 8
    st = _strides(D)
    total = prod(d + 1 for d in D)
    pos_buf = bytearray(total * nb)
    neg_buf = bytearray(total * nb)
    for e, c in zip(P.lex_exponents(degs), vec):
        c = int(c)
        if not c:
            continue
        at = sum(x * s for x, s in zip(e, st)) * nb
        buf = pos_buf if c > 0 else neg_buf
        buf[at:at + nb] = abs(c).to_bytes(nb, "little")
    return int.from_bytes(pos_buf, "little") - int.from_bytes(neg_buf, "little")


def unpack(x: int, D: Sequence[int], b: int) -> List[int]:
    """Balanced base-2^b digits of x at the places of the box prod [0, D_v],
    returned as the lex coefficient vector of that box."""
    assert b % 8 == 0
    nb = b // 8
    total = prod(d + 1 for d in D)
    raw = x.to_bytes((total + 1) * nb, "little", signed=True)
    half = 1 << (b - 1)
    full = 1 << b
    out = [0] * total
    carry = 0
    for i in range(total):
        u = int.from_bytes(raw[i * nb:(i + 1) * nb], "little") + carry
        if u >= half:
            u -= full
            carry = 1
        else:
            carry = 0
        out[i] = u
    top = int.from_bytes(raw[total * nb:], "little") + carry
    if top % full:
        raise ArithmeticError("packed value does not fit the degree box")
    # positions are mixed-radix in (D_1+1, ..., D_k+1) with x_k fastest, which
    # is exactly the lex order of the box: no reordering needed.
    return out


def digit_bits(coeffs, degs: Sequence[int]) -> int:
    """b: a multiple of 8 with 2^(b-1) > 2 * (Hadamard bound on |coeff|)."""
    bsq = hadamard_bound_sq(coeffs, degs)
    bound = _isqrt_ceil(bsq)
    b = bound.bit_length() + 2
    return (b + 7) // 8 * 8


def _isqrt_ceil(x: int) -> int:
    from math import isqrt
    r = isqrt(x)
    return r if r * r == x else r + 1


def det_packed(coeffs, degs: Sequence[int]) -> List[int]:
    """O2: the determinant as the lex coefficient vector of the box
    prod [0, D_v], D_v = n * d_v, via integer Bareiss on packed entries."""
    n = len(coeffs)
    D = det_degree_bound(n, degs)
    b = digit_bits(coeffs, degs)
    M = [[pack(coeffs[i][j], degs, D, b) for j in range(n)] for i in range(n)]
    return unpack(det_bareiss_int(M), D, b)


def det_poly_dense(coeffs, degs: Sequence[int]) -> List[int]:
    """O1 with dense output over the box prod [0, n*d_v] (for comparison)."""
    n = len(coeffs)
    k = len(degs)
    M = P.matrix_from_dense(coeffs, degs)
    det = det_bareiss_poly(M, k)
    return P.to_dense(det, det_degree_bound(n, degs))


def det_bareiss(M) -> "np.ndarray":
    """O1 on a matrix given entry by entry, returning the determinant as a
    dense object array of Python ints with shape (D_1+1, ..., D_k+1), index
    (e_1, ..., e_k) the exponent vector (D_v = n * d_v, Sec. 2).

    Each entry of ``M`` is either a dict {exponent tuple: int} or an integer
    array of shape (d_1+1, ..., d_k+1) indexed by the exponent vector; the
    number of variables k and the degrees d_v are read off the entries (the
    largest exponent of x_v over all entries)."""
    import numpy as np
    n = len(M)
    k = 0
    for row in M:
        for e in row:
            if isinstance(e, dict):
                k = max(k, max((len(x) for x in e), default=0))
            else:
                k = max(k, np.asarray(e).ndim)
    k = max(k, 1)
    polys = []
    for row in M:
        prow = []
        for e in row:
            if isinstance(e, dict):
                prow.append({tuple(x) + (0,) * (k - len(x)): int(c) for x, c in e.items() if c})
            else:
                a = np.asarray(e)
                a = a.reshape(a.shape + (1,) * (k - a.ndim))
                prow.append({tuple(int(i) for i in idx): int(c) for idx, c in np.ndenumerate(a) if c})
        polys.append(prow)
    degs = [max((x[v] for row in polys for e in row for x in e), default=0) for v in range(k)]
    D = det_degree_bound(n, degs)
    out = np.zeros([d + 1 for d in D], dtype=object)
    det = det_bareiss_poly(polys, k) if n else P.const(1, k)
    for x, c in det.items():
        out[x] = c
    return out
