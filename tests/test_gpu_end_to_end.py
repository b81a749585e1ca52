"""Exact determinants end to end on the GPU against the CPU oracle
(bit-exact: the output is a list of integers)."""
import hashlib
import json
import os

import numpy as np
import pytest

from helpers import ROOT, ensure_lib
from oracle import bareiss, certificate, plan as oplan
from oracle import poly as P_
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def det(pm, **kw):
    from paper_2010_12117_gb300.pipeline import determinant
    return determinant(pm.coeffs, pm.degs, **kw)


@pytest.mark.parametrize("seed", range(5))
def test_dense_4x4_xy(seed):
    pm = synth.dense_4x4(seed)
    got = det(pm)
    assert got.coeffs == bareiss.det_poly_dense(pm.coeffs.tolist(), pm.degs)
    assert got.coeffs == bareiss.det_packed(pm.coeffs.tolist(), pm.degs)


@pytest.mark.parametrize("seed", range(3))
def test_sylvester_16_x(seed):
    pm = synth.sylvester_16(seed)
    got = det(pm)
    assert got.P >= 10
    assert got.coeffs == bareiss.det_packed(pm.coeffs.tolist(), pm.degs)


@pytest.mark.parametrize("n,degs,density", [(5, (2, 2, 2), 0.3), (6, (1, 2, 1), 0.5),
                                            (3, (3, 3, 3), 1.0), (7, (1, 1), 0.3)])
def test_small_multivariate(n, degs, density):
    rng = np.random.default_rng(n * 31 + len(degs))
    pm = synth.random_matrix(rng, n, degs, density, -128, 128)
    got = det(pm)
    assert got.coeffs == bareiss.det_packed(pm.coeffs.tolist(), pm.degs)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _digest(coeffs):
    return hashlib.sha256(",".join(str(int(c)) for c in coeffs).encode()).hexdigest()


@pytest.mark.parametrize("nprimes", [None, 20])
def test_sparse_12x12_xyz_full_size(nprimes):
    """Full workload (12x12 over Z[x,y,z], 64^3 grid): the whole output
    against the oracle's stored digest, sampled coefficients one by one, and
    a Schwartz-Zippel certificate; with the Hadamard prime count and with 20
    primes (extra primes must not change the result)."""
    g = _golden("sparse_12x12_xyz_seed0.json")
    pm = synth.sparse_12x12_xyz(0)
    got = det(pm, nprimes=nprimes)
    assert len(got.coeffs) == g["coefficients"]
    for i, v in g["samples"].items():
        assert got.coeffs[int(i)] == int(v), i
    assert _digest(got.coeffs) == g["sha256"]
    if nprimes is None:
        assert certificate.check(pm.coeffs.tolist(), pm.degs, got.coeffs, got.D, trials=8)
    else:
        assert got.P == 20


@pytest.mark.parametrize("maker", [lambda: synth.dense_4x4(3), lambda: synth.sylvester_16(4),
                                   lambda: synth.random_matrix(np.random.default_rng(2), 5, (2, 1, 2),
                                                               0.5, -99, 100)])
def test_full_grid_and_node_grid_agree_with_the_oracle(maker):
    """The paper's full power-of-two grid with inverse NTT and the node grid
    with inverse Vandermonde give the oracle's determinant."""
    pm = maker()
    want = bareiss.det_packed(pm.coeffs.tolist(), pm.degs)
    assert det(pm, full_grid=True).coeffs == want
    assert det(pm, full_grid=False).coeffs == want


def test_extra_primes_and_larger_degree_box_do_not_change_the_result():
    rng = np.random.default_rng(77)
    pm = synth.random_matrix(rng, 5, (2, 1), 0.6, -1000, 1000)
    base = det(pm)
    more = det(pm, nprimes=base.P + 3)
    assert more.coeffs == base.coeffs
    # the same polynomials declared with one more degree per variable: a
    # bigger grid (oversize N_v) and a bigger output box, same determinant
    big = (3, 2)
    c2 = np.zeros((5, 5, 4 * 3), dtype=np.int64)
    for i in range(5):
        for j in range(5):
            poly = P_.from_dense(pm.coeffs[i, j].tolist(), pm.degs)
            c2[i, j] = P_.to_dense(poly, big)
    pm2 = synth.PolyMatrix(5, big, c2)
    got2 = det(pm2)
    want = P_.from_dense(base.coeffs, base.D)
    assert P_.from_dense(got2.coeffs, got2.D) == want


def test_edge_cases():
    k = 2
    # 1x1: the entry itself
    pm = synth.PolyMatrix(1, (3, 2), np.arange(12, dtype=np.int64).reshape(1, 1, 12) - 6)
    assert det(pm).coeffs == pm.coeffs[0, 0].tolist()
    # zero matrix
    z = synth.PolyMatrix(4, (1, 1), np.zeros((4, 4, 4), dtype=np.int64))
    assert not any(det(z).coeffs)
    # rank-deficient polynomial matrix: row 2 = x * row 0 + row 1
    rng = np.random.default_rng(8)
    pm = synth.random_matrix(rng, 4, (2, 2), 0.8, -9, 10)
    M = P_.matrix_from_dense(pm.coeffs.tolist(), pm.degs)
    x = P_.var(0, k)
    M[2] = [P_.add(P_.mul(x, M[0][j]), M[1][j]) for j in range(4)]
    degs = (3, 2)
    c = np.array([[P_.to_dense(M[i][j], degs) for j in range(4)] for i in range(4)], dtype=np.int64)
    assert not any(det(synth.PolyMatrix(4, degs, c)).coeffs)
    # anti-diagonal (every pivot needs the search): det = sign * product
    a = np.zeros((6, 6, 2), dtype=np.int64)
    for i in range(6):
        a[i, 5 - i] = [i + 1, 1]  # (i+1) + x
    got = det(synth.PolyMatrix(6, (1,), a)).coeffs
    want = P_.const(-1, 1)  # reversal of 6 rows: 3 swaps
    for i in range(6):
        want = P_.mul(want, {(0,): i + 1, (1,): 1})
    assert P_.from_dense(got, (6,)) == want


def test_vandermonde_and_resultant_pins_on_gpu():
    """The closed forms of the oracle pins, now through the CUDA path."""
    k = 2
    x, y = P_.var(0, k), P_.var(1, k)
    n = 6
    ts = [P_.add(P_.add(x, P_.scale(y, i)), P_.const(c, k)) for i, c in enumerate([3, -1, 4, 1, -5, 9])]
    M = [[P_.power(ts[i], j, k) for j in range(n)] for i in range(n)]
    want = P_.const(1, k)
    for i in range(n):
        for j in range(i + 1, n):
            want = P_.mul(want, P_.sub(ts[j], ts[i]))
    degs = (n - 1, n - 1)
    c = np.array([[P_.to_dense(M[i][j], degs) for j in range(n)] for i in range(n)], dtype=np.int64)
    got = det(synth.PolyMatrix(n, degs, c))
    assert P_.from_dense(got.coeffs, got.D) == want


def test_batched_members_certified():
    """Members of the batched workload through the plain path: bit-exact
    against O2 when small, Schwartz-Zippel certified otherwise."""
    ms = synth.batched(0, 12)
    for pm in ms:
        got = det(pm)
        cost = pm.n ** 3 * np.prod([pm.n * d + 1 for d in pm.degs])
        if cost < 3e6:
            assert got.coeffs == bareiss.det_packed(pm.coeffs.tolist(), pm.degs), pm.name
        else:
            assert certificate.check(pm.coeffs.tolist(), pm.degs, got.coeffs, got.D, trials=8), pm.name


def test_six_variables_and_long_univariate_grids():
    """The widest shapes the plan takes: six variables (the maximum), and one
    variable with 6001 nodes (a 2x2 matrix of degree-3000 polynomials: 750
    whole cosets of the 8th roots plus one node) against the oracle."""
    rng = np.random.default_rng(606)
    pm = synth.random_matrix(rng, 2, (1, 1, 1, 1, 1, 1), 0.8, -50, 50)
    got = det(pm)
    assert got.coeffs == bareiss.det_packed(pm.coeffs.tolist(), pm.degs)
    pm = synth.random_matrix(rng, 2, (3000,), 1.0, -1000, 1000)
    got = det(pm)
    assert got.coeffs == bareiss.det_packed(pm.coeffs.tolist(), pm.degs)
    # the full grid (8192 nodes, inverse NTT) gives the same
    assert det(pm, full_grid=True).coeffs == got.coeffs
