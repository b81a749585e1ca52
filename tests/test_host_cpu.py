"""Host logic of the batched form, on CPU: the per-job variable order and
the transpositions of input and output it implies, checked against the
oracle's determinant (det commutes with renaming the variables)."""
import numpy as np
import pytest

from oracle import bareiss
from oracle.plan import det_degree_bound
from paper_2010_12117_gb300 import synth
from paper_2010_12117_gb300.binding import BATCH_MATERIALIZE_N
from paper_2010_12117_gb300.runner import permute_coeffs, unpermute_output, variable_order


def test_variable_order_rule():
    # fused orders (n below the threshold): the sorted order reversed, so the
    # lowest degree is last (and ties come out reversed)
    assert variable_order(5, (3, 1, 2)) == [0, 2, 1]
    assert variable_order(5, (2, 2, 1)) == [1, 0, 2]
    # materialized orders: lowest degree first
    n = BATCH_MATERIALIZE_N
    assert variable_order(n, (3, 1, 2)) == [1, 2, 0]
    assert variable_order(n, (2, 2, 1)) == [2, 0, 1]
    assert variable_order(7, (4,)) == [0]


@pytest.mark.parametrize("n,degs,seed", [(3, (2, 1), 1), (4, (1, 3), 2), (3, (1, 2, 1), 3),
                                         (2, (3, 1, 2), 4), (BATCH_MATERIALIZE_N - 11, (2, 0, 1), 5)])
def test_permuted_determinant_transposes_back(n, degs, seed):
    rng = np.random.default_rng(seed)
    pm = synth.random_matrix(rng, n, degs, 0.8, -20, 20)
    want = bareiss.det_packed(pm.coeffs.tolist(), pm.degs)
    for order in (variable_order(n, degs), list(range(len(degs)))[::-1]):
        pdegs = tuple(degs[v] for v in order)
        pc = permute_coeffs(pm.coeffs, degs, order)
        got = bareiss.det_packed(pc.tolist(), pdegs)
        box = tuple(D + 1 for D in det_degree_bound(n, pdegs))
        assert unpermute_output(got, order, box) == want, (n, degs, order)


def test_identity_order_is_untouched():
    vals = [5, -3, 0, 7]
    assert unpermute_output(vals, [0, 1], (2, 2)) == vals
    # a transposition of a 2 x 2 box swaps the off-diagonal coefficients
    assert unpermute_output(vals, [1, 0], (2, 2)) == [5, 0, -3, 7]
