"""polydet_interp_static: interpolation for callers that cannot allocate
device memory when they need the result (inside a global-mode stream
capture, under a foreign allocator that owns the device memory, or in a
loop that must not stall on cudaMalloc/cudaFree).  Its scratch is a fixed
array inside the library, so it must give exactly what polydet_interp gives
with a caller workspace - on consecutive calls that reuse that array - and
must refuse requests larger than the array without touching anything.

This file is named to be collected last: the other GPU tests have run by the
time it does, and it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from helpers import ensure_lib
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _detvals(pm, P):
    """Determinant values at every node for the first P primes (plain path)."""
    from paper_2010_12117_gb300.binding import Plan
    pl = Plan(pm.n, pm.degs, P)
    c = torch.from_numpy(pm.coeffs.astype(np.int32).reshape(-1)).cuda()
    ev = torch.empty(P * pm.n * pm.n * pl.G, dtype=torch.int32, device="cuda")
    dv = torch.empty(P * pl.G, dtype=torch.int32, device="cuda")
    pl.eval(c, 0, P, ev, pl.workspace(P))
    pl.condense(ev, 0, P, dv)
    torch.cuda.synchronize()
    return pl, dv


def _call_static(pl, dv, lo, hi, out):
    """Through the C ABI directly."""
    from paper_2010_12117_gb300 import binding
    L = binding.lib()
    return L.polydet_interp_static(pl._h, ctypes.c_void_p(dv.data_ptr()), lo, hi,
                                   ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_scratch_interp_equals_workspace_interp_on_consecutive_calls():
    from paper_2010_12117_gb300.binding import OK, as_u32
    # three variables: every interpolation pass but the last uses the scratch
    pm = synth.sparse_12x12_xyz(1)
    P = 3
    pl, dv = _detvals(pm, P)
    assert pl.interp_ws_words * P <= 4 * 1024 * 1024
    want = torch.empty(P * pl.C, dtype=torch.int32, device="cuda")
    pl.interp(dv, 0, P, want, pl.workspace(P))
    assert pl.sync_status() == 0
    # first call: all primes; second call: a sub-range whose detvals start at
    # prime 1, reusing the array the first call left behind
    got = torch.full((P * pl.C,), -1, dtype=torch.int32, device="cuda")
    assert _call_static(pl, dv, 0, P, got) == OK
    assert pl.sync_status() == 0
    assert np.array_equal(as_u32(got), as_u32(want))
    got2 = torch.full((2 * pl.C,), -1, dtype=torch.int32, device="cuda")
    assert _call_static(pl, dv[pl.G:], 1, P, got2) == OK
    assert pl.sync_status() == 0
    assert np.array_equal(as_u32(got2), as_u32(want)[pl.C:])


def test_static_scratch_interp_two_calls_on_a_second_shape():
    """Two more calls in a row on another plan (two variables) after the
    three-variable calls have used the array."""
    from paper_2010_12117_gb300.binding import as_u32
    rng = np.random.default_rng(3)
    pm = synth.random_matrix(rng, 9, (3, 2), 0.6, -500, 500)
    P = 4
    pl, dv = _detvals(pm, P)
    want = torch.empty(P * pl.C, dtype=torch.int32, device="cuda")
    pl.interp(dv, 0, P, want, pl.workspace(P))
    for _ in range(2):
        got = torch.zeros(P * pl.C, dtype=torch.int32, device="cuda")
        pl.interp_static(dv, 0, P, got)
        torch.cuda.synchronize()
        assert pl.sync_status() == 0
        assert np.array_equal(as_u32(got), as_u32(want))


def test_static_scratch_refuses_oversized_requests():
    from paper_2010_12117_gb300.binding import ETOOBIG, Plan
    # 24x24 over Z[x,y,z] with degrees 4: 2^20 nodes per prime; each prime
    # needs ~1.6M words of scratch, so 3 primes exceed the 4M-word array
    pl = Plan(24, (4, 4, 4), 3)
    assert pl.interp_ws_words * 3 > 4 * 1024 * 1024
    dv = torch.zeros(3 * pl.G, dtype=torch.int32, device="cuda")
    out = torch.full((3 * pl.C,), 7, dtype=torch.int32, device="cuda")
    assert _call_static(pl, dv, 0, 3, out) == ETOOBIG
    torch.cuda.synchronize()
    assert int((out != 7).sum()) == 0  # nothing was written
