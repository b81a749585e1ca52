"""Stage-by-stage parity of the CUDA kernels with the CPU oracle, through the
C ABI.  Integer work: every comparison is bit-exact."""
import random
from math import prod

import numpy as np
import pytest

from helpers import ensure_lib, evals_tensor, random_residue_mats
from oracle import modular, plan as oplan
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def Plan(n, degs, P, full_grid=False):
    from paper_2010_12117_gb300.binding import Plan as _P
    return _P(n, degs, P, full_grid=full_grid)


def u32(t):
    from paper_2010_12117_gb300.binding import as_u32
    return as_u32(t)


def test_plan_constants_match_oracle():
    pl = Plan(12, (3, 3, 3), 5)
    assert pl.primes == modular.ntt_primes()[:5]
    assert pl.D == (36, 36, 36) and pl.N == (64, 64, 64) and pl.M == (37, 37, 37)
    assert pl.G == 37 ** 3 and pl.C == 37 ** 3 and pl.E == 64
    full = Plan(12, (3, 3, 3), 5, full_grid=True)
    assert full.M == (64, 64, 64) and full.G == 64 ** 3 and full.full_grid
    for q, p in enumerate(pl.primes):
        for v, N in enumerate(pl.N):
            assert pl.roots[q][v] == modular.root_of_unity(p, N)
    assert pl.W == oplan.output_words(pl.primes)


@pytest.mark.parametrize("n,degs,P,sample,full", [
    (4, (2, 2), 2, None, False),          # dense 4x4 workload, every node
    (4, (2, 2), 2, None, True),           # ... on the full power-of-two grid
    (3, (2, 0, 1), 2, None, False),       # a variable of degree 0 (one node)
    (3, (2, 0, 1), 2, None, True),
    (16, (6,), 3, None, False),           # Sylvester-sized univariate
    (2, (7, 5), 2, None, False),          # 8 coefficients: the LP = 8 coset kernel
    (5, (3, 1, 2), 2, 300, True),         # trivariate, sampled nodes
    (12, (3, 3, 3), 1, 40, False),        # 12x12 trivariate grid, sampled
    (12, (3, 3, 3), 1, 40, True),
])
def test_eval_matches_direct_evaluation(n, degs, P, sample, full):
    rng = np.random.default_rng(n + 7 * P)
    pm = synth.random_matrix(rng, n, degs, 0.7, -(2 ** 31), 2 ** 31)
    pm.coeffs[0, 0, 0] = -(2 ** 31)  # extreme int32 values
    pm.coeffs[0, 0, -1] = 2 ** 31 - 1
    pl = Plan(n, degs, P, full_grid=full)
    coeffs = torch.from_numpy(pm.coeffs.astype(np.int32).reshape(-1)).cuda()
    evals = torch.empty(P * n * n * pl.G, dtype=torch.int32, device="cuda")
    pl.eval(coeffs, 0, P, evals, pl.workspace(P))
    torch.cuda.synchronize()
    got = u32(evals).reshape(P, n * n, pl.G)
    nodes = range(pl.G) if sample is None else sorted(set(
        [0, pl.G - 1] + [int(x) for x in rng.integers(0, pl.G, sample)]))
    entries = range(n * n) if n * n <= 16 or sample is None else \
        sorted(set([0, n * n - 1] + [int(x) for x in rng.integers(0, n * n, 12)]))
    for q in range(P):
        p = pl.primes[q]
        ws = pl.roots[q]
        for e in entries:
            vec = pm.coeffs.reshape(n * n, -1)[e].tolist()
            for g in nodes:
                idx = modular.grid_index(g, pl.M)
                ex = [pl.node_exps[v][i] for v, i in enumerate(idx)]  # the plan's node order
                assert int(got[q, e, g]) == modular.eval_point(vec, degs, ex, ws, p), (q, e, g)


def test_eval_prime_range_offsets():
    """A range [lo, hi) writes slot 0 for prime lo."""
    n, degs = 4, (2, 2)
    rng = np.random.default_rng(3)
    pm = synth.random_matrix(rng, n, degs, 1.0, -10, 11)
    pl = Plan(n, degs, 4)
    coeffs = torch.from_numpy(pm.coeffs.astype(np.int32).reshape(-1)).cuda()
    full = torch.empty(4 * n * n * pl.G, dtype=torch.int32, device="cuda")
    part = torch.empty(2 * n * n * pl.G, dtype=torch.int32, device="cuda")
    pl.eval(coeffs, 0, 4, full, pl.workspace(4))
    pl.eval(coeffs, 2, 4, part, pl.workspace(2))
    torch.cuda.synchronize()
    assert np.array_equal(u32(full)[2 * n * n * pl.G:], u32(part))


def _special_matrices(n, p, rng):
    """Matrices that force the pivot search or are singular."""
    mats = []
    I = np.eye(n, dtype=np.uint64)
    mats.append(I)                                   # identity
    perm = np.eye(n, dtype=np.uint64)[rng.permutation(n)]
    mats.append(perm)                                # permutation: every pivot searched
    z = np.zeros((n, n), dtype=np.uint64)
    mats.append(z)                                   # zero matrix
    r = rng.integers(0, p, (n, n), dtype=np.uint64)
    if n > 1:
        r2 = r.copy()
        r2[n - 1] = r2[0]
        mats.append(r2)                              # duplicate row: det 0
        r3 = r.copy()
        r3[:, 0] = 0
        r3[n - 1, 0] = 5
        mats.append(r3)                              # only the last row can pivot column 0
        r4 = r.copy()
        r4[: n // 2, : n // 2] = 0
        mats.append(r4)                              # zero leading block
        r5 = np.triu(r)
        mats.append(r5)                              # triangular
        r6 = r.copy()
        r6[:, n // 2] = 0
        mats.append(r6)                              # zero column: det 0
    mats.append(np.full((n, n), p - 1, dtype=np.uint64))  # all -1: rank 1
    return mats


@pytest.mark.parametrize("n", list(range(1, 33)))
def test_condense_matches_gaussian_elimination(n):
    """Every matrix order 1..32 (each kernel instantiation), random residues,
    sparse residues and matrices that need the pivot search."""
    rng = np.random.default_rng(500 + n)
    d = max(1, 128 // n)  # G between 128 and 512 nodes
    P = 2
    pl = Plan(n, (d,), P)
    G = pl.G
    mats = random_residue_mats(rng, P, G, n, pl.primes)
    # sparse residues in a quarter of the nodes
    for q in range(P):
        sp = random_residue_mats(rng, 1, G // 4, n, pl.primes[q:q + 1], zero_frac=0.6)[0]
        mats[q, : G // 4] = sp
        for s, M in enumerate(_special_matrices(n, pl.primes[q], rng)):
            mats[q, G // 4 + s] = M % pl.primes[q]
    evals = evals_tensor(mats, G)
    det = torch.empty(P * G, dtype=torch.int32, device="cuda")
    pl.condense(evals, 0, P, det)
    torch.cuda.synchronize()
    got = u32(det).reshape(P, G)
    check = sorted(set(range(0, G // 4, max(1, G // 64))) | set(range(G // 4, G // 4 + 12)) |
                   set(int(x) for x in rng.integers(0, G, 24)) | {G - 1})
    if n <= 6:
        check = range(G)
    for q in range(P):
        p = pl.primes[q]
        for g in check:
            want = modular.det_mod_p(mats[q, g].astype(object).tolist(), p)
            assert int(got[q, g]) == want, (n, q, g)


@pytest.mark.parametrize("full,degs", [(False, (2, 2)), (True, (2, 2)), (False, (1, 2, 1)),
                                        (False, (5,))])
def test_interp_round_trip_against_oracle(full, degs):
    """Interpolation of the oracle's evaluations of a random polynomial of
    bounded degree returns its coefficients, with a clean status - on the node
    grid (inverse Vandermonde) and on the full grid (inverse NTT)."""
    n, P = 4, 2
    pl = Plan(n, degs, P, full_grid=full)
    rng = random.Random(17)
    det_vals = np.empty((P, pl.G), dtype=np.uint64)
    want = []
    for q in range(P):
        p = pl.primes[q]
        vec = [rng.randrange(p) for _ in range(pl.C)]
        want.append(vec)
        det_vals[q] = [modular.eval_point(vec, pl.D, [pl.node_exps[v][i] for v, i in
                                                      enumerate(modular.grid_index(g, pl.M))],
                                          pl.roots[q], p) for g in range(pl.G)]
    dv = torch.from_numpy(det_vals.astype(np.uint32).view(np.int32).reshape(-1)).cuda()
    res = torch.empty(P * pl.C, dtype=torch.int32, device="cuda")
    pl.interp(dv, 0, P, res, pl.workspace(P))
    assert pl.sync_status() == 0
    got = u32(res).reshape(P, pl.C)
    for q in range(P):
        assert got[q].tolist() == want[q]
    # and against the oracle's interpolation of the same values directly
    if full:
        box, clean = modular.interp_grid(det_vals[0].tolist(), pl.N, pl.roots[0], pl.primes[0], pl.D)
        assert clean and box == want[0]
    else:
        assert modular.interp_nodes(det_vals[0].tolist(), pl.M, pl.roots[0], pl.primes[0],
                                    pl.node_exps) == want[0]


@pytest.mark.parametrize("n,degs", [(4, (1, 2, 3)), (24, (3, 4)), (1, (7,)), (3, (0, 2))])
def test_node_order_is_whole_cosets(n, degs):
    """The node grid visits distinct powers of w_v coset by coset: node k is
    w^(k // L + (N/L) (k mod L)) with L = pow2 >= min(d_v + 1, 8); the full
    grid is natural."""
    pl = Plan(n, degs, 2)
    for v, d in enumerate(degs):
        L = 1
        while L < min(d + 1, 8):
            L *= 2
        N = pl.N[v]
        want = [k // L + (N // L) * (k % L) for k in range(pl.M[v])]
        assert pl.node_exps[v] == want
        assert len(set(want)) == pl.M[v] and max(want) < N
    full = Plan(n, degs, 2, full_grid=True)
    assert full.node_exps == [list(range(N)) for N in full.N]


def test_interp_flags_a_degree_bound_violation():
    """Values that are not those of a polynomial within the box leave a
    nonzero tail: the status word reports it (no fault, no abort)."""
    from paper_2010_12117_gb300.binding import EBOUND, lib
    n, degs, P = 2, (1, 1), 1  # D = (2, 2) inside the 4 x 4 grid: a 7-value tail
    pl = Plan(n, degs, P, full_grid=True)
    assert pl.C < pl.G
    rng = np.random.default_rng(5)
    vals = rng.integers(0, pl.primes[0], pl.G, dtype=np.uint64).astype(np.uint32)
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    res = torch.empty(pl.C, dtype=torch.int32, device="cuda")
    pl.interp(dv, 0, 1, res, pl.workspace(1))
    assert pl.sync_status() & 1
    assert pl.sync_status() == 0  # reading clears it
    # the kept coefficients still equal the oracle's inverse DFT of those values
    box, clean = modular.interp_grid(vals.tolist(), pl.N, pl.roots[0], pl.primes[0], pl.D)
    assert not clean and u32(res).tolist() == box


@pytest.mark.parametrize("P", [1, 2, 5, 11, 20, 24, 40, 91])
def test_crt_matches_garner(P):
    d = 700 if P < 40 else 120  # C = d + 1: not a multiple of the CTA size
    pl = Plan(1, (d,), P)
    C = pl.C
    rng = random.Random(P)
    M = prod(pl.primes)
    xs = [rng.randrange(-(M // 2), M // 2 + 1) for _ in range(C)]
    for j, X in enumerate([0, 1, -1, M // 2, -(M // 2), M // 2 - 1, -(M // 2) + 1]):
        xs[j] = X
    res = np.array([[X % p for X in xs] for p in pl.primes], dtype=np.uint64).astype(np.uint32)
    rd = torch.from_numpy(res.view(np.int32).reshape(-1)).cuda()
    limbs = torch.empty(C * pl.W, dtype=torch.int32, device="cuda")
    pl.crt(rd, limbs)
    torch.cuda.synchronize()
    from paper_2010_12117_gb300.binding import limbs_to_ints
    got = limbs_to_ints(u32(limbs).reshape(C, pl.W), pl.W)
    for j in range(C):
        assert got[j] == modular.garner(res[:, j].tolist(), pl.primes) == xs[j], j
    # the raw words are the oracle's two's complement limbs
    assert u32(limbs).reshape(C, pl.W)[3].tolist() == modular.to_limbs(xs[3], pl.W)


def test_invalid_arguments_are_rejected():
    from paper_2010_12117_gb300.binding import EINVAL, PolydetError
    pl = Plan(4, (2, 2), 2)
    buf = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        pl.eval(buf, 0, 2, buf, pl.workspace(2))  # too small
    with pytest.raises(ValueError):
        big0 = torch.empty(2 * 16 * pl.G, dtype=torch.int32, device="cuda")
        pl.eval(torch.zeros(16 * 9, dtype=torch.int32, device="cuda"), 0, 2, big0)  # no workspace
    big = torch.empty(4 * 16 * pl.G, dtype=torch.int32, device="cuda")
    with pytest.raises(PolydetError) as ei:
        pl.condense(big, 1, 1, big)  # empty range
    assert ei.value.code == EINVAL
    with pytest.raises(PolydetError):
        pl.interp(big, 0, 3, big, pl.workspace(3))  # beyond P
    with pytest.raises(PolydetError):
        Plan(33, (1,), 2)
    with pytest.raises(PolydetError):
        Plan(4, (3000,), 2)  # N_v beyond 8192


def test_integer_pipe_probes_report_ordered_rates():
    """The probes behind the condensation's roofline: every rate positive and
    finite, and the element updates ordered by their work (a plain IMAD, then
    the single-step update of two products, the two-step element of three and
    the three-step element of four, each under one REDC)."""
    import math
    from paper_2010_12117_gb300.binding import probe_int_peaks
    imad, one, two, three = probe_int_peaks()
    for r in (imad, one, two, three):
        assert r > 0 and math.isfinite(r)
    assert imad > one > two > three


def test_shape_cache_eviction_and_clear_keep_results_exact():
    """More distinct shapes than the cache keeps (256 unused): the oldest
    shapes' tables go back to the library's pool, a plan of such a shape is
    built again, and after polydet_plan_cache_clear every table is rebuilt;
    the determinant of a small job stays the oracle's throughout."""
    from oracle import bareiss
    from paper_2010_12117_gb300.binding import Plan as _P, lib
    from paper_2010_12117_gb300.pipeline import determinant
    pm = synth.dense_4x4(0)
    want = bareiss.det_packed(pm.coeffs.tolist(), pm.degs)
    assert determinant(pm.coeffs, pm.degs).coeffs == want
    shapes = [(n, (d,), P) for n in range(1, 7) for d in range(1, 6) for P in range(2, 12)]
    assert len(shapes) > 256
    for n, degs, P in shapes:
        _P(n, degs, P).close()
    assert determinant(pm.coeffs, pm.degs).coeffs == want
    pl = _P(*shapes[0])  # evicted by now: built again
    assert pl.P == shapes[0][2]
    pl.close()
    assert lib().polydet_plan_cache_clear() == 0
    assert determinant(pm.coeffs, pm.degs).coeffs == want
