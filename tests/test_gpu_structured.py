"""Structured and large-degree inputs through the CUDA path: evaluation of
distinct entries only (entry map), the determinant degree bound from the
entries' degrees, and evaluation + condensation streamed slab by slab
through a bounded workspace.  Every result is checked against the oracle
(O2 bit-exact where it finishes, the limb certificate otherwise) or against
the plain path, which the other tests tie to the oracle."""
import numpy as np
import pytest

from helpers import ensure_lib
from oracle import bareiss, certificate, plan as oplan
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def det(pm, **kw):
    from paper_2010_12117_gb300.pipeline import determinant
    return determinant(pm.coeffs, pm.degs, **kw)


def _embed(vals, D_small, D_big):
    """Coefficients over the box prod [0, D_small] placed in prod [0, D_big]."""
    out = np.zeros([d + 1 for d in D_big], dtype=object)
    out[tuple(slice(0, d + 1) for d in D_small)] = np.array(vals, dtype=object).reshape([d + 1 for d in D_small])
    return out.reshape(-1).tolist()


def _with_repeats(rng, n, degs, U, pzero, lo=-500, hi=500):
    """n x n matrix whose entries are drawn from U distinct polynomials, with
    a fraction pzero of zero entries."""
    E = int(np.prod([d + 1 for d in degs]))
    base = rng.integers(lo, hi, (U, E))
    pick = rng.integers(0, U, (n, n))
    c = base[pick].astype(np.int64)
    c[rng.random((n, n)) < pzero] = 0
    return synth.PolyMatrix(n, tuple(degs), c)


def test_sylvester_with_entry_map_equals_oracle():
    """The 16 x 16 Sylvester workload: 18 distinct entries (f_0..f_8,
    g_0..g_8) and 256 - 144 zero entries; only 19 entries per prime are
    evaluated, the result is the oracle's."""
    from paper_2010_12117_gb300.binding import Plan, unique_entries
    pm = synth.sylvester_16(3)
    m, U, _ = unique_entries(pm.coeffs)
    assert U == 18
    pl = Plan(16, pm.degs, 2)
    pl.set_entry_map(m, U)
    assert pl.entries == 19 and pl.items == 18
    pl.close()
    got = det(pm, unique_entries=True)
    assert got.coeffs == bareiss.det_packed(pm.coeffs.tolist(), pm.degs)


@pytest.mark.parametrize("n,degs,U,pz", [(5, (3,), 4, 0.2), (8, (2, 1), 6, 0.3), (12, (1, 1, 1), 9, 0.1),
                                         (17, (2,), 30, 0.4), (23, (1, 1), 12, 0.0)])
def test_entry_map_equals_plain(n, degs, U, pz):
    rng = np.random.default_rng(n * 7 + U)
    pm = _with_repeats(rng, n, degs, U, pz)
    want = det(pm)
    assert det(pm, unique_entries=True).coeffs == want.coeffs
    if n ** 3 * np.prod([n * d + 1 for d in degs]) < 2e6:
        assert want.coeffs == bareiss.det_packed(pm.coeffs.tolist(), pm.degs)


def test_entry_map_zero_matrix_and_single_entry():
    pm = synth.PolyMatrix(6, (2,), np.zeros((6, 6, 3), dtype=np.int64))
    assert not any(det(pm, unique_entries=True).coeffs)
    c = np.zeros((4, 4, 3), dtype=np.int64)
    for i in range(4):
        c[i, i] = [1, 2, 1]  # (1 + x)^2 on the diagonal: det = (1 + x)^8
    got = det(synth.PolyMatrix(4, (2,), c), unique_entries=True)
    from math import comb
    assert got.coeffs == [comb(8, i) for i in range(9)]


@pytest.mark.parametrize("m,l,df,dg", [(3, 2, (2, 1), (1, 3)), (4, 3, (1, 1, 1), (2, 1, 0)),
                                       (2, 2, (3, 2, 1, 1), (1, 1, 2, 1))])
def test_tight_degree_bound_equals_oracle(m, l, df, dg):
    """Sylvester matrices over several variables with the assignment degree
    bound: the output box shrinks to the resultant bound, and the
    coefficients are the oracle's (which outside the box are zero)."""
    rng = np.random.default_rng(m * 10 + l)
    pm = synth.sylvester(rng, m, l, df, dg, 0.6, -50, 50)
    got = det(pm, tight_degrees=True)
    want_box = oplan.assignment_degree_bound(oplan.entry_degrees(pm.coeffs.tolist(), pm.degs), len(pm.degs))
    assert got.D == want_box
    full = bareiss.det_packed(pm.coeffs.tolist(), pm.degs)
    assert _embed(got.coeffs, got.D, oplan.det_degree_bound(pm.n, pm.degs)) == full
    assert det(pm, tight_degrees=True, unique_entries=True).coeffs == got.coeffs


@pytest.mark.parametrize("full_grid", [False, True])
@pytest.mark.parametrize("unique", [False, True])
def test_streamed_equals_plain(full_grid, unique):
    """Evaluation + condensation streamed through a workspace that holds
    only a few x_1 nodes at a time (several slabs and a ragged last one)."""
    rng = np.random.default_rng(17 + full_grid + 2 * unique)
    cases = [_with_repeats(rng, 9, (3, 5, 2), 7, 0.2), synth.random_matrix(rng, 13, (4, 2), 0.6, -900, 900),
             synth.random_matrix(rng, 6, (9,), 0.8, -9, 9), synth.random_matrix(rng, 4, (1, 1, 1, 2), 0.7, -9, 9)]
    for pm in cases:
        want = det(pm, full_grid=full_grid)
        G_bytes = 4 * pm.n ** 2 * np.prod([pm.n * d + 1 for d in pm.degs])
        for budget in (int(G_bytes // 5), int(G_bytes // 2)):
            got = det(pm, full_grid=full_grid, unique_entries=unique, streamed=True, budget_bytes=budget)
            assert got.coeffs == want.coeffs, (pm.n, pm.degs, budget)


def test_streamed_slabs_directly():
    """polydet_eval_condense with workspaces of 1, 2 and 3 cosets of x_1 per
    slab gives the determinant values polydet_eval + polydet_condense_batch
    give, for every prime of a range."""
    from paper_2010_12117_gb300.binding import Plan, as_u32
    rng = np.random.default_rng(23)
    pm = synth.random_matrix(rng, 10, (3, 6), 0.7, -99, 99)  # x_1 cosets of 4 nodes, M_1 = 31
    P = 3
    pl = Plan(10, pm.degs, P)
    c = torch.from_numpy(pm.coeffs.astype(np.int32).reshape(-1)).cuda()
    ev = torch.empty(P * pl.entries * pl.G, dtype=torch.int32, device="cuda")
    want = torch.empty(P * pl.G, dtype=torch.int32, device="cuda")
    pl.eval(c, 0, P, ev, pl.workspace(P))
    pl.condense(ev, 0, P, want)
    for rows in (1, 4, 8, 12, 31):
        ws = torch.empty(pl.stream_ws_words(rows), dtype=torch.int32, device="cuda")
        got = torch.full((P * pl.G,), -1, dtype=torch.int32, device="cuda")
        pl.eval_condense(c, 0, P, got, ws)
        torch.cuda.synchronize()
        assert np.array_equal(as_u32(got), as_u32(want)), rows
    too_small = torch.empty(max(1, pl.stream_ws_words(1) - 1), dtype=torch.int32, device="cuda")
    from paper_2010_12117_gb300.binding import PolydetError
    with pytest.raises(PolydetError):
        pl.eval_condense(c, 0, P, want, too_small)
    assert pl.sync_status() == 0
    pl.close()


def test_four_variable_sylvester_shrunk_is_exact():
    """A small matrix of the four-variable Sylvester shape through the
    streamed path with the entry map and the tight bound: bit-exact against
    O2."""
    rng = np.random.default_rng(5)
    pm = synth.sylvester(rng, 3, 2, (3, 2, 2, 1), (2, 2, 1, 1), 0.3, -128, 128)
    got = det(pm, tight_degrees=True, unique_entries=True, streamed=True, budget_bytes=1 << 20)
    full = bareiss.det_packed(pm.coeffs.tolist(), pm.degs)
    assert _embed(got.coeffs, got.D, oplan.det_degree_bound(pm.n, pm.degs)) == full


def test_four_variable_sylvester_full_size_certified():
    """The 15 x 15 Sylvester matrix over Z[x1..x4] with determinant degrees
    (298, 171, 119, 45) - 2.8e8 nodes and coefficients per prime - streamed
    within a 24 GB workspace budget with the entry map: certified from its
    limbs at 8 random points mod 2^31 - 1."""
    from paper_2010_12117_gb300.pipeline import determinant
    pm = synth.sylvester_15_four_vars(0)
    got = determinant(pm.coeffs, pm.degs, tight_degrees=True, unique_entries=True,
                      streamed=True, budget_bytes=24 << 30, as_ints=False)
    assert got.D == (298, 171, 119, 45)
    assert certificate.check_limbs(pm.coeffs, pm.degs, got.limbs, got.D, trials=8)
