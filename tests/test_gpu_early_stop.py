"""Early termination: the digit check of polydet_crt_check against the
oracle's definition of a stable lift, and determinants taken with early stop
against the oracle and the full prime count."""
import numpy as np
import pytest

from helpers import ensure_lib
from oracle import bareiss, modular
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def test_crt_check_matches_the_stable_lift_definition():
    """Coefficients of every size from 0 to beyond M_P / 2 (both signs, and
    the boundary values +-(M_i - 1) / 2 and +-(M_i + 1) / 2): after each
    prime i the device flag is set exactly when the oracle finds some
    coefficient whose lift over i primes differs from the lift over i + 1."""
    from math import prod
    from paper_2010_12117_gb300.binding import Plan
    P = 9
    C = 4096
    pl = Plan(1, (C - 1,), P)
    assert pl.C == C
    ps = pl.primes
    rng = np.random.default_rng(8)
    for trial in range(3):
        top = int(rng.integers(1, P))  # values need about `top` primes at most
        vals = []
        for k in range(C):
            b = int(rng.integers(0, 31 * top + 1))
            v = int.from_bytes(rng.bytes(32 * P // 8 + 8), "little") % (1 << b) if b else 0
            vals.append(-v if rng.random() < 0.5 else v)
        for i in range(1, P):
            Mi = prod(ps[:i])
            vals[(7 * i) % C] = (Mi - 1) // 2
            vals[(7 * i + 1) % C] = -((Mi - 1) // 2)
        res = np.array([[v % p for v in vals] for p in ps], dtype=np.uint64).astype(np.uint32)
        r = torch.from_numpy(res.view(np.int32).reshape(-1)).cuda()
        digits = torch.empty(P * C, dtype=torch.int32, device="cuda")
        flag = torch.zeros(1, dtype=torch.int32, device="cuda")
        for i in range(1, P):
            flag.zero_()
            pl.crt_check(r, digits, i, flag)
            want = not all(modular.lift_is_stable([v % p for p in ps[:i + 1]], ps) for v in vals)
            assert bool(int(flag.item())) == want, (trial, i)
    # the digits left behind are Garner's
    d = digits.cpu().numpy().view(np.uint32).reshape(P, C)
    for k in range(0, C, 97):
        assert d[:, k].tolist() == modular.mixed_radix_digits([int(x) for x in res[:, k]], ps), k
    pl.close()


@pytest.mark.parametrize("n,degs,ddegs", [(6, (2, 1), (1, 1)), (9, (3,), (1,)), (5, (1, 1, 1), (1, 0, 1))])
def test_early_stop_on_small_determinants_is_exact(n, degs, ddegs):
    rng = np.random.default_rng(n)
    pm = synth.small_det_matrix(rng, n, degs, ddegs, mixes=n)
    from paper_2010_12117_gb300.pipeline import determinant
    got = determinant(pm.coeffs, pm.degs, early_stop=True)
    assert got.coeffs == bareiss.det_packed(pm.coeffs.tolist(), pm.degs)
    assert got.P < got.primes_bound


def test_early_stop_agrees_with_the_full_count():
    """Singular and generic matrices: early stop gives the full-count
    result (a zero determinant after two primes)."""
    from paper_2010_12117_gb300.pipeline import determinant
    rng = np.random.default_rng(12)
    pm = synth.random_matrix(rng, 7, (2, 2), 0.8, -3000, 3000)
    c = pm.coeffs.copy()
    c[5] = c[2]  # duplicate row
    sing = determinant(c, pm.degs, early_stop=True)
    assert not any(sing.coeffs) and sing.P == 2
    for pm in synth.batched(3, 6):
        full = determinant(pm.coeffs, pm.degs)
        early = determinant(pm.coeffs, pm.degs, early_stop=True)
        assert early.coeffs == full.coeffs, pm.name
        assert early.P <= full.P


def test_early_stop_streamed_with_entry_map():
    from paper_2010_12117_gb300.pipeline import determinant
    rng = np.random.default_rng(14)
    pm = synth.small_det_matrix(rng, 12, (2, 2), (1, 1), mixes=12)
    want = determinant(pm.coeffs, pm.degs)
    got = determinant(pm.coeffs, pm.degs, early_stop=True, streamed=True, unique_entries=True,
                      budget_bytes=1 << 22)
    assert got.coeffs == want.coeffs and got.P < want.P
