"""Seeded synthetic inputs: polynomial matrices over Z[x1..xk].

This module only draws random numbers and lays them out; it holds none of the
determinant method's arithmetic.  Both the CUDA path and the CPU oracle are fed
from it, so it imports neither.

Layout of a matrix (the dense coefficient encoding of Sec. 2 of the paper):
``coeffs[i, j, :]`` holds the coefficients of entry (i, j) for the exponent
vectors (e1, ..., ek), 0 <= e_v <= d_v, in lex order with x1 slowest and xk
fastest.  For F = 1 + 2x + 3xy + 4x^2 + 5y^2 with d = (2, 2) this is
[1, 0, 5, 2, 3, 0, 4, 0, 0], the example printed in Sec. 2.

Draw order (numpy ``default_rng(seed)``, PCG64), per workload:

* ``dense_4x4``: one ``integers(-10, 11, (4, 4, 9))`` call.
* ``sylvester_16``: f then g, each ``integers(-2**15, 2**15, (9, 7))`` indexed
  [power of y][power of x]; the 16x16 Sylvester matrix in y is then laid out.
* ``sylvester`` / ``sylvester_15_four_vars``: see ``sylvester``.
* ``small_det_matrix``: see its docstring.
* ``sparse_12x12_xyz``: ``random((12, 12, 64)) < 0.3`` (monomial mask) then
  ``integers(-128, 128, (12, 12, 64))`` (values); masked-out values become 0.
* ``batched``: per matrix, in order: n = integers(4, 25); k = integers(1, 4);
  d = integers(1, 5, k); density = uniform(0.3, 1.0); then mask and int16
  values as above.
* ``served_stream``: per job: inter-arrival gap = exponential(1/rate); u =
  random(); if u < 0.05 a large 32x32 job over Z[x, y] with d = (6, 6), dense
  int16, else one ``batched`` draw.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

INT16_LO, INT16_HI = -(2 ** 15), 2 ** 15


@dataclass
class PolyMatrix:
    """An n x n matrix over Z[x1..xk] in the dense lex encoding.

    ``coeffs`` is int64 with shape (n, n, prod(d_v + 1)).
    """

    n: int
    degs: Tuple[int, ...]
    coeffs: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nvars(self) -> int:
        return len(self.degs)

    @property
    def terms(self) -> int:
        return int(np.prod([d + 1 for d in self.degs]))

    def entry(self, i: int, j: int) -> np.ndarray:
        """Coefficients of entry (i, j) shaped (d_1+1, ..., d_k+1)."""
        return self.coeffs[i, j].reshape([d + 1 for d in self.degs])


def random_matrix(rng: np.random.Generator, n: int, degs: Sequence[int],
                  density: float, lo: int, hi: int, name: str = "") -> PolyMatrix:
    """Each monomial of each entry is kept with probability ``density``;
    kept monomials get a value uniform in [lo, hi) (a zero draw stays zero)."""
    degs = tuple(int(d) for d in degs)
    t = int(np.prod([d + 1 for d in degs]))
    mask = rng.random((n, n, t)) < density
    vals = rng.integers(lo, hi, (n, n, t))
    coeffs = np.where(mask, vals, 0).astype(np.int64)
    return PolyMatrix(n, degs, coeffs, name=name, meta={"density": float(density)})


def dense_4x4(seed: int) -> PolyMatrix:
    """4x4 over Z[x, y], every entry dense with degree <= 2 in each variable,
    coefficients uniform in [-10, 10]."""
    rng = np.random.default_rng(seed)
    c = rng.integers(-10, 11, (4, 4, 9)).astype(np.int64)
    return PolyMatrix(4, (2, 2), c, name=f"dense_4x4_xy/seed{seed}")


def sylvester_layout(f: np.ndarray, g: np.ndarray) -> PolyMatrix:
    """Sylvester matrix in y of f = sum_i f[i](x) y^i and g = sum_i g[i](x) y^i.

    ``f`` and ``g`` are [power of y][power of x] integer arrays with the same
    x-degree bound.  Row r < deg g holds f's coefficients from the leading one
    down, shifted right by r; row deg g + r holds g's, shifted right by r.
    """
    m = f.shape[0] - 1
    l = g.shape[0] - 1
    n = m + l
    t = f.shape[1]
    c = np.zeros((n, n, t), dtype=np.int64)
    for r in range(l):
        for s in range(m + 1):
            c[r, r + s] = f[m - s]
    for r in range(m):
        for s in range(l + 1):
            c[l + r, r + s] = g[l - s]
    return PolyMatrix(n, (t - 1,), c)


def sylvester(rng: np.random.Generator, m: int, l: int, degs_f: Sequence[int],
              degs_g: Sequence[int], density: float, lo: int, hi: int) -> PolyMatrix:
    """(m + l) x (m + l) Sylvester matrix in y of f = sum_{i<=m} f_i y^i and
    g = sum_{i<=l} g_i y^i with f_i, g_i in Z[x1..xk] of degree <= degs_f
    (degs_g) in x_v.  Draws, f's coefficients i = 0..m then g's: a monomial
    mask ``random(E) < density`` and values ``integers(lo, hi, E)`` over the
    polynomial's own degree box, then for each v with a positive degree the
    pure power x_v^d_v gets ``integers(lo, hi)`` (1 where that draw is 0), so
    that every f_i, g_i reaches its degree bound in every variable.  Entries
    are encoded over the box of the larger bounds."""
    degs_f = tuple(int(d) for d in degs_f)
    degs_g = tuple(int(d) for d in degs_g)
    box = tuple(max(a, b) for a, b in zip(degs_f, degs_g))

    def draw(degs):
        shape = tuple(d + 1 for d in degs)
        E = int(np.prod(shape))
        mask = rng.random(E) < density
        vals = np.where(mask, rng.integers(lo, hi, E), 0).reshape(shape)
        for v, d in enumerate(degs):
            if d > 0:
                idx = tuple(d if u == v else 0 for u in range(len(degs)))
                x = int(rng.integers(lo, hi))
                vals[idx] = x if x != 0 else 1
        out = np.zeros(tuple(b + 1 for b in box), dtype=np.int64)
        out[tuple(slice(0, d + 1) for d in degs)] = vals
        return out.reshape(-1)

    f = np.stack([draw(degs_f) for _ in range(m + 1)])
    g = np.stack([draw(degs_g) for _ in range(l + 1)])
    pm = sylvester_layout(f, g)
    pm.degs = box
    pm.name = f"sylvester_{m + l}_k{len(box)}"
    pm.meta = {"m": m, "l": l, "degs_f": degs_f, "degs_g": degs_g}
    return pm


def sylvester_15_four_vars(seed: int, density: float = 0.01) -> PolyMatrix:
    """15 x 15 Sylvester matrix in y of f (degree 8 in y) and g (degree 7)
    over Z[x1, x2, x3, x4], coefficient polynomials of degree (22, 13, 9, 3)
    for f and (18, 10, 7, 3) for g, int8 coefficients: its determinant (the
    resultant) has degree at most 7 * 22 + 8 * 18 = 298, 171, 119 and 45 in
    the four variables, the shape of the harmonic-elimination matrix of
    Sec. 6 (whose polynomials the paper does not give)."""
    rng = np.random.default_rng(seed)
    pm = sylvester(rng, 8, 7, (22, 13, 9, 3), (18, 10, 7, 3), density, -128, 128)
    pm.name = f"sylvester_15_x1x2x3x4/seed{seed}"
    return pm


def small_det_matrix(rng: np.random.Generator, n: int, degs: Sequence[int], diag_degs: Sequence[int],
                     mixes: int = 0) -> PolyMatrix:
    """An n x n matrix over Z[x1..xk] whose determinant is far smaller than
    its Hadamard bound.  Draws, in order: entries strictly above the diagonal
    dense int16 over the box ``degs``; diagonal entries over the box
    ``diag_degs`` with coefficients in [-2, 2] and a constant term in {1, 2}
    (entries below the diagonal are zero); then ``mixes`` integer row
    operations row_i += c row_j (i != j, c in [-3, 3]) and a random
    permutation of the rows and one of the columns.  The determinant is,
    up to sign, the product of the diagonal entries drawn."""
    degs = tuple(int(d) for d in degs)
    shape = tuple(d + 1 for d in degs)
    E = int(np.prod(shape))
    c = np.zeros((n, n, E), dtype=np.int64)
    for i in range(n):
        for j in range(i + 1, n):
            c[i, j] = rng.integers(INT16_LO, INT16_HI, E)
    for i in range(n):
        dsh = tuple(int(d) + 1 for d in diag_degs)
        d = rng.integers(-2, 3, dsh)
        d.flat[0] = int(rng.integers(1, 3))
        box = np.zeros(shape, dtype=np.int64)
        box[tuple(slice(0, k) for k in dsh)] = d
        c[i, i] = box.reshape(-1)
    for _ in range(mixes):
        i, j = (int(x) for x in rng.choice(n, 2, replace=False))
        c[i] += int(rng.integers(-3, 4)) * c[j]
    c = c[rng.permutation(n)][:, rng.permutation(n)]
    if np.abs(c).max() >= 2 ** 31:
        raise ValueError("mixed entries no longer fit in int32")
    return PolyMatrix(n, degs, c, name=f"small_det_{n}x{n}_k{len(degs)}")


def sylvester_16(seed: int) -> PolyMatrix:
    """16x16 Sylvester matrix of f, g in Z[x][y], both of degree 8 in y, with
    coefficient polynomials in x of degree <= 6 and int16 coefficients."""
    rng = np.random.default_rng(seed)
    f = rng.integers(INT16_LO, INT16_HI, (9, 7)).astype(np.int64)
    g = rng.integers(INT16_LO, INT16_HI, (9, 7)).astype(np.int64)
    pm = sylvester_layout(f, g)
    pm.name = f"sylvester_16_x/seed{seed}"
    pm.meta = {"f": f, "g": g}
    return pm


def sparse_12x12_xyz(seed: int) -> PolyMatrix:
    """12x12 over Z[x, y, z], degree <= 3 per variable, 30% of the monomials
    nonzero, int8 coefficients uniform in [-128, 127]."""
    rng = np.random.default_rng(seed)
    pm = random_matrix(rng, 12, (3, 3, 3), 0.3, -128, 128)
    pm.name = f"sparse_12x12_xyz/seed{seed}"
    return pm


def batched_member(rng: np.random.Generator, idx: int = 0) -> PolyMatrix:
    n = int(rng.integers(4, 25))
    k = int(rng.integers(1, 4))
    degs = tuple(int(d) for d in rng.integers(1, 5, k))
    density = float(rng.uniform(0.3, 1.0))
    pm = random_matrix(rng, n, degs, density, INT16_LO, INT16_HI)
    pm.name = f"batched[{idx}]"
    return pm


def batched(seed: int, count: int = 256) -> List[PolyMatrix]:
    """``count`` matrices with n ~ U[4, 24], k ~ U{1, 2, 3}, d_v ~ U[1, 4],
    density ~ U[0.3, 1.0], int16 coefficients."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        pm = batched_member(rng, i)
        pm.name = f"batched/seed{seed}[{i}]"
        out.append(pm)
    return out


def large_32x32_xy(rng: np.random.Generator, idx: int = 0) -> PolyMatrix:
    pm = random_matrix(rng, 32, (6, 6), 1.0, INT16_LO, INT16_HI)
    pm.name = f"large_32x32_xy[{idx}]"
    return pm


@dataclass
class Arrival:
    t: float
    job: PolyMatrix


def served_stream(seed: int, njobs: int, rate: float,
                  large_frac: float = 0.05) -> List[Arrival]:
    """Poisson arrivals at ``rate`` jobs/s: the batched distribution plus a
    ``large_frac`` share of 32x32 jobs over Z[x, y] with degree <= 6."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(njobs):
        t += float(rng.exponential(1.0 / rate))
        if rng.random() < large_frac:
            job = large_32x32_xy(rng, i)
        else:
            job = batched_member(rng, i)
        job.name = f"served/seed{seed}[{i}]"
        out.append(Arrival(t, job))
    return out


WORKLOADS = {
    "dense_4x4_xy": dense_4x4,
    "sylvester_16_x": sylvester_16,
    "sparse_12x12_xyz": sparse_12x12_xyz,
}


def gen_config(i: int, seed: int, **kw):
    """The seeded input of one of the five workloads, by index: 0 the dense
    4x4 over Z[x, y], 1 the 16x16 Sylvester matrix, 2 the sparse 12x12 over
    Z[x, y, z] (each a PolyMatrix), 3 the batched list of ``count`` (default
    256) matrices, 4 the served stream of ``njobs`` (default 300) Poisson
    arrivals at ``rate`` jobs/s (default 700)."""
    if i == 0:
        return dense_4x4(seed)
    if i == 1:
        return sylvester_16(seed)
    if i == 2:
        return sparse_12x12_xyz(seed)
    if i == 3:
        return batched(seed, kw.get("count", 256))
    if i == 4:
        return served_stream(seed, kw.get("njobs", 300), kw.get("rate", 700.0),
                             kw.get("large_frac", 0.05))
    raise ValueError(f"no workload with index {i}")
