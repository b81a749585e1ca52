"""Multivariate integer polynomials for the oracle (plain Python ints).

A polynomial in k variables is a dict mapping an exponent tuple (e1..ek) to a
nonzero int.  Python compares tuples lexicographically, so ``max(p)`` is the
leading monomial in lex order with x1 most significant, the order of the
coefficient encoding of Sec. 2.
"""
from __future__ import annotations

from itertools import product
from typing import Dict, Iterable, List, Sequence, Tuple

Exp = Tuple[int, ...]
Poly = Dict[Exp, int]


def zero() -> Poly:
    return {}


def const(c: int, k: int) -> Poly:
    return {(0,) * k: int(c)} if c else {}


def var(v: int, k: int) -> Poly:
    e = [0] * k
    e[v] = 1
    return {tuple(e): 1}


def add(a: Poly, b: Poly) -> Poly:
    r = dict(a)
    for e, c in b.items():
        s = r.get(e, 0) + c
        if s:
            r[e] = s
        else:
            r.pop(e, None)
    return r


def neg(a: Poly) -> Poly:
    return {e: -c for e, c in a.items()}


def sub(a: Poly, b: Poly) -> Poly:
    return add(a, neg(b))


def scale(a: Poly, s: int) -> Poly:
    if s == 0:
        return {}
    return {e: c * s for e, c in a.items()}


def mul(a: Poly, b: Poly) -> Poly:
    """Schoolbook product: every term of a times every term of b."""
    r: Poly = {}
    for ea, ca in a.items():
        for eb, cb in b.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            s = r.get(e, 0) + ca * cb
            if s:
                r[e] = s
            else:
                r.pop(e, None)
    return r


def divexact(a: Poly, b: Poly) -> Poly:
    """Quotient q with a = q*b, for b dividing a exactly in Z[x1..xk].

    Textbook multivariate division by the lex-leading term: repeatedly divide
    the leading term of the remainder by the leading term of b.  Exactness of
    every step is asserted (the remainder must reach zero).
    """
    if not b:
        raise ZeroDivisionError("division by the zero polynomial")
    lt_b = max(b)
    lc_b = b[lt_b]
    q: Poly = {}
    r = dict(a)
    while r:
        e = max(r)
        c = r[e]
        m = tuple(x - y for x, y in zip(e, lt_b))
        if min(m) < 0 or c % lc_b:
            raise ArithmeticError("division is not exact")
        qc = c // lc_b
        q[m] = qc
        for eb, cb in b.items():
            t = tuple(x + y for x, y in zip(m, eb))
            s = r.get(t, 0) - qc * cb
            if s:
                r[t] = s
            else:
                r.pop(t, None)
    return q


def power(a: Poly, n: int, k: int) -> Poly:
    r = const(1, k)
    for _ in range(n):
        r = mul(r, a)
    return r


def degrees(a: Poly, k: int) -> Tuple[int, ...]:
    """Per-variable degree; -1 for a variable that does not occur (or a=0)."""
    out = [-1] * k
    for e in a:
        for v in range(k):
            out[v] = max(out[v], e[v])
    return tuple(out)


def evaluate_mod(a: Poly, point: Sequence[int], q: int) -> int:
    """a(point) mod q, term by term."""
    s = 0
    for e, c in a.items():
        t = c
        for x, ev in zip(point, e):
            t = t * pow(x, ev, q) % q
        s += t
    return s % q


# ---------------------------------------------------------------------------
# Dense lex encoding (Sec. 2): exponent vectors 0 <= e_v <= d_v, x1 slowest.
# ---------------------------------------------------------------------------

def lex_exponents(degs: Sequence[int]) -> List[Exp]:
    """All exponent vectors of the box prod [0, d_v] in lex order, x1 slowest."""
    return [tuple(e) for e in product(*[range(d + 1) for d in degs])]


def from_dense(vec: Iterable[int], degs: Sequence[int]) -> Poly:
    """Inverse of the Sec. 2 encoding: a flat lex coefficient vector to a dict."""
    r: Poly = {}
    for e, c in zip(lex_exponents(degs), vec):
        c = int(c)
        if c:
            r[e] = c
    return r


def to_dense(a: Poly, degs: Sequence[int]) -> List[int]:
    """The Sec. 2 encoding: coefficients of the box prod [0, d_v], lex order.

    Raises if a has a term outside the box.
    """
    for e in a:
        if any(x > d for x, d in zip(e, degs)):
            raise ValueError(f"term {e} outside degree box {tuple(degs)}")
    return [a.get(e, 0) for e in lex_exponents(degs)]


def matrix_from_dense(coeffs, degs: Sequence[int]) -> List[List[Poly]]:
    """coeffs[i][j][:] (lex vectors) to an n x n list of dict polynomials."""
    n = len(coeffs)
    return [[from_dense(coeffs[i][j], degs) for j in range(n)] for i in range(n)]


def l1_norm(a: Poly) -> int:
    return sum(abs(c) for c in a.values())
