"""Stage-by-stage references of the modular method (Sec. 2-3), on Python ints.

Each function is the plain definition of what one stage computes, with no
fast transform, blocking or reordering:

* primes of the form c * 2^q + 1 (Eq. 1) and their roots of unity;
* evaluation of an entry on the grid of roots (what the multivariate Stockham
  FFT of Sec. 3.1 / Algorithm 2 produces) as the direct sum over monomials;
* the determinant mod p at one node (Sec. 3.2 / Algorithm 3) by Gaussian
  elimination with modular inverses;
* interpolation (Sec. 3.3) as the inverse DFT with the 1/N factor;
* mixed-radix (Garner) reconstruction (Sec. 3.4 / Algorithm 4) and the
  textbook CRT formula beside it.
"""
from __future__ import annotations

from itertools import product
from math import prod
from typing import Optional, Dict, List, Sequence, Tuple

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Miller-Rabin with the first twelve prime bases (deterministic for
    n < 3.3e24, far above the 31-bit primes used here)."""
    if n < 2:
        return False
    for q in _MR_BASES:
        if n % q == 0:
            return n == q
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


NTT_Q = 20  # every prime admits 2^20-th roots of unity


# The order in which the method takes the primes is free (the output does not
# depend on it).  The table lists those up to this value first: a sum of three
# products of residues below p, reduced once mod p, stays unambiguous in 32 bits
# only up to it, and the GPU condensation relies on that.
FOLD3_MAX = 1865126253


def ntt_primes() -> List[int]:
    """All primes p = c * 2^20 + 1 (Eq. 1 with q = 20) in (2^30, 2^31): those
    up to FOLD3_MAX largest first, then the others largest first."""
    out = []
    for c in range((2 ** 31 - 1) >> NTT_Q, (2 ** 30) >> NTT_Q, -1):
        p = (c << NTT_Q) + 1
        if 2 ** 30 < p < 2 ** 31 and is_prime(p):
            out.append(p)
    return [p for p in out if p <= FOLD3_MAX] + [p for p in out if p > FOLD3_MAX]


def prime_factors(n: int) -> List[int]:
    fs, d = [], 2
    while d * d <= n:
        if n % d == 0:
            fs.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        fs.append(n)
    return fs


def primitive_root(p: int) -> int:
    """Least generator of (Z/pZ)^*."""
    fs = prime_factors(p - 1)
    g = 2
    while any(pow(g, (p - 1) // q, p) == 1 for q in fs):
        g += 1
    return g


def root_of_unity(p: int, N: int) -> int:
    """omega = g^((p-1)/N): a principal N-th root of unity mod p (N | p-1)."""
    if (p - 1) % N:
        raise ValueError("N does not divide p - 1")
    return pow(primitive_root(p), (p - 1) // N, p)


def grid_index(g: int, Ns: Sequence[int]) -> Tuple[int, ...]:
    """Flat grid index (lex, x1 slowest) -> (i1, ..., ik)."""
    idx = []
    for N in reversed(Ns):
        idx.append(g % N)
        g //= N
    return tuple(reversed(idx))


def eval_point(vec: Sequence[int], degs: Sequence[int], idx: Sequence[int],
               omegas: Sequence[int], p: int) -> int:
    """One entry (lex coefficient vector) at the node x_v = omega_v^(i_v):
    sum_e c_e prod_v omega_v^(i_v e_v) mod p."""
    s = 0
    for e, c in zip(product(*[range(d + 1) for d in degs]), vec):
        c = int(c)
        if not c:
            continue
        t = c % p
        for w, i, ev in zip(omegas, idx, e):
            t = t * pow(w, i * ev, p) % p
        s += t
    return s % p


def eval_grid(vec, degs, Ns, omegas, p) -> List[int]:
    """The entry at every node of the grid prod [0, N_v), lex order."""
    return [eval_point(vec, degs, grid_index(g, Ns), omegas, p)
            for g in range(prod(Ns))]


def det_mod_p(A: Sequence[Sequence[int]], p: int) -> int:
    """Determinant over F_p: Gaussian elimination, first nonzero pivot in the
    column, row swaps flip the sign, det = sign * product of pivots."""
    M = [[int(x) % p for x in row] for row in A]
    n = len(M)
    det = 1
    for c in range(n):
        r = next((i for i in range(c, n) if M[i][c]), None)
        if r is None:
            return 0
        if r != c:
            M[c], M[r] = M[r], M[c]
            det = -det
        piv = M[c][c]
        det = det * piv % p
        inv = pow(piv, p - 2, p)
        for i in range(c + 1, n):
            f = M[i][c] * inv % p
            if f:
                for j in range(c, n):
                    M[i][j] = (M[i][j] - f * M[c][j]) % p
    return det % p


def interp_grid(values: Sequence[int], Ns: Sequence[int], omegas: Sequence[int],
                p: int, D: Sequence[int]) -> Tuple[List[int], bool]:
    """Inverse DFT with the 1/N factor (Sec. 3.3): coefficient of x^e is
    prod_v N_v^{-1} * sum_i values[i] prod_v omega_v^(-i_v e_v).

    Returns the coefficients of the box prod [0, D_v] (lex) and whether every
    coefficient with some e_v in (D_v, N_v) is zero, as it must be when D_v
    bounds the degree.
    """
    inv_n = pow(prod(Ns), p - 2, p)
    inv_w = [pow(w, p - 2, p) for w in omegas]
    G = prod(Ns)
    idxs = [grid_index(g, Ns) for g in range(G)]
    box: List[int] = []
    clean = True
    for e in product(*[range(N) for N in Ns]):
        s = 0
        for g in range(G):
            t = values[g]
            for w, i, ev in zip(inv_w, idxs[g], e):
                t = t * pow(w, i * ev, p) % p
            s += t
        c = s * inv_n % p
        if all(ev <= dv for ev, dv in zip(e, D)):
            box.append(c)
        elif c:
            clean = False
    return box, clean


def solve_mod_p(A: Sequence[Sequence[int]], b: Sequence[int], p: int) -> List[int]:
    """x with A x = b over F_p (A square, invertible): Gauss-Jordan."""
    n = len(A)
    M = [[int(v) % p for v in row] + [int(bb) % p] for row, bb in zip(A, b)]
    for c in range(n):
        r = next(i for i in range(c, n) if M[i][c])
        M[c], M[r] = M[r], M[c]
        inv = pow(M[c][c], p - 2, p)
        M[c] = [v * inv % p for v in M[c]]
        for i in range(n):
            if i != c and M[i][c]:
                f = M[i][c]
                M[i] = [(vi - f * vc) % p for vi, vc in zip(M[i], M[c])]
    return [M[i][n] for i in range(n)]


def interp_nodes(values: Sequence[int], Ms: Sequence[int], omegas: Sequence[int],
                 p: int, exps: Optional[Sequence[Sequence[int]]] = None) -> List[int]:
    """Interpolation through the node grid x_v = omega_v^(s_v(i)), 0 <= i < M_v,
    with s_v(i) = i unless ``exps[v]`` lists the exponents s_v (any M_v
    distinct powers; Sec. 3.3: the polynomial of degree < M_v in each variable
    through M_v distinct nodes is unique): one Vandermonde system V c = y per
    line, variable by variable.  ``values`` lex over the grid; returns lex
    coefficients of the box prod [0, M_v)."""
    k = len(Ms)
    cur = [int(v) % p for v in values]
    for v in range(k - 1, -1, -1):
        m = Ms[v]
        s = list(range(m)) if exps is None else [int(x) for x in exps[v]]
        V = [[pow(omegas[v], s[i] * e, p) for e in range(m)] for i in range(m)]
        inner = prod(Ms[v + 1:])
        outer = prod(Ms[:v])
        nxt = [0] * len(cur)
        for a in range(outer):
            for b in range(inner):
                idx = [(a * m + i) * inner + b for i in range(m)]
                coef = solve_mod_p(V, [cur[t] for t in idx], p)
                for e, t in enumerate(idx):
                    nxt[t] = coef[e]
        cur = nxt
    return cur


def mixed_radix_digits(xs: Sequence[int], primes: Sequence[int]) -> List[int]:
    """Garner / MRC digits (Sec. 3.4, reading of Eq. for alpha_i):
    X = sum_i alpha_i prod_{l<i} p_l with 0 <= alpha_i < p_i and
    X = x_i mod p_i.  alpha_i = (x_i - sum_{j<i} alpha_j prod_{l<j} p_l) *
    (prod_{l<i} p_l)^{-1} mod p_i."""
    alphas: List[int] = []
    for i, (x, p) in enumerate(zip(xs, primes)):
        s = 0
        m = 1
        for j in range(i):
            s += alphas[j] * m
            m *= primes[j]
        c_i = pow(m % p, p - 2, p)
        alphas.append((x - s) * c_i % p)
    return alphas


def from_mixed_radix(alphas: Sequence[int], primes: Sequence[int]) -> int:
    """Horner form X = a_0 + p_0 (a_1 + p_1 (a_2 + ...))."""
    X = 0
    for a, p in zip(reversed(alphas), reversed(primes)):
        X = X * p + a
    return X


def symmetric_lift(X: int, M: int) -> int:
    """The representative of X mod M in (-M/2, M/2) (M odd, so no tie)."""
    X %= M
    return X - M if X > M // 2 else X


def garner(xs: Sequence[int], primes: Sequence[int]) -> int:
    """Signed integer with the given residues, via mixed-radix digits."""
    return symmetric_lift(from_mixed_radix(mixed_radix_digits(xs, primes), primes),
                          prod(primes))


def crt_direct(xs: Sequence[int], primes: Sequence[int]) -> int:
    """Textbook CRT: X = sum_i x_i (M/p_i) ((M/p_i)^{-1} mod p_i) mod M,
    then the symmetric lift.  Independent of the mixed-radix route."""
    M = prod(primes)
    X = 0
    for x, p in zip(xs, primes):
        Mi = M // p
        X += x * Mi * pow(Mi % p, p - 2, p)
    return symmetric_lift(X, M)


def to_limbs(X: int, W: int) -> List[int]:
    """Two's complement of X in W little-endian 32-bit words."""
    if not -(1 << (32 * W - 1)) <= X < (1 << (32 * W - 1)):
        raise OverflowError("value does not fit in W words")
    u = X % (1 << (32 * W))
    return [(u >> (32 * i)) & 0xFFFFFFFF for i in range(W)]


def count_ntt_primes_after(start: int, count: int, qs: Sequence[int]) -> Dict[int, int]:
    """Among the first ``count`` primes strictly above ``start``, how many
    satisfy 2^q | p - 1, for each q (the quantity tabulated in Sec. 4.2).
    The function is pinned (hand-counted cases and an independent count);
    only its comparison with the printed table is unpinned, because the
    paper's exact counting rule is not recoverable from its text."""
    out = {q: 0 for q in qs}
    p = start
    found = 0
    while found < count:
        p += 1
        if is_prime(p):
            found += 1
            for q in qs:
                if (p - 1) % (1 << q) == 0:
                    out[q] += 1
    return out


def lift_is_stable(xs: Sequence[int], primes: Sequence[int]) -> bool:
    """Early termination's test, by its plain definition: the symmetric lift
    of the residues ``xs[:i]`` over the first i primes equals the symmetric
    lift of ``xs[:i + 1]`` over the first i + 1 (i = len(xs) - 1 >= 1)."""
    i = len(xs) - 1
    a = symmetric_lift(crt_direct(xs[:i], primes[:i]), prod(primes[:i]))
    b = symmetric_lift(crt_direct(xs, primes[:i + 1]), prod(primes[:i + 1]))
    return a == b
