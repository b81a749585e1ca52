"""The batched form (fused last-variable evaluation + condensation, one
persistent kernel per matrix order, CUDA graph) against the plain per-matrix
GPU form and the CPU oracle: identical integers."""
import numpy as np
import pytest

from helpers import ensure_lib
from oracle import bareiss, certificate
from oracle import poly as P_
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def batched_results(mats, tune=False, graph=False, replays=1, full_grid=False, modes=None,
                    chunk_words=None):
    from paper_2010_12117_gb300.runner import BatchedRunner
    st = torch.cuda.Stream()
    r = BatchedRunner(mats, tune=tune, stream=st, full_grid=full_grid)
    if modes is not None:
        r.set_modes(modes)
    if chunk_words is not None:
        r.set_chunk_words(chunk_words)
    r.upload(st)
    if graph:
        r.capture(st)
    for _ in range(replays):
        r.compute(st)
    r.download(st)
    st.synchronize()
    r.check_status(st)
    out = r.results()
    r.close()
    return out


def plain(pm):
    from paper_2010_12117_gb300.pipeline import determinant
    return determinant(pm.coeffs, pm.degs).coeffs


def _mixed():
    rng = np.random.default_rng(4242)
    mats = []
    for n, degs, dens in [(1, (3,), 1.0), (2, (1, 1), 1.0), (3, (2, 0, 1), 0.8), (4, (2, 2), 0.5),
                          (5, (1, 2, 1), 0.4), (6, (4,), 0.3), (7, (1, 1), 0.6), (8, (2,), 1.0),
                          (9, (1, 1, 1), 0.3), (10, (1,), 0.5), (11, (1, 2), 0.3), (12, (1, 1, 1), 0.3),
                          (13, (2,), 0.6), (14, (1,), 1.0), (16, (1, 1), 0.3), (17, (1,), 0.7),
                          (20, (1, 1), 0.3), (21, (2,), 0.5), (24, (1,), 0.4), (25, (1,), 1.0),
                          (28, (1,), 0.3), (32, (1,), 0.5), (4, (7,), 1.0), (6, (1, 7), 0.5)]:
        mats.append(synth.random_matrix(rng, n, degs, dens, -300, 300))
    return mats


def test_mixed_orders_match_plain_and_oracle():
    mats = _mixed()
    got = batched_results(mats)
    for pm, g in zip(mats, got):
        assert g == plain(pm), (pm.n, pm.degs)
        cost = pm.n ** 3 * np.prod([pm.n * d + 1 for d in pm.degs])
        if cost < 2e6:
            assert g == bareiss.det_packed(pm.coeffs.tolist(), pm.degs), (pm.n, pm.degs)


def test_fused_and_materialized_modes_agree():
    """Every order fused, every order materialized, and the default split:
    the same integers (and equal to the plain form)."""
    from paper_2010_12117_gb300.binding import BATCH_FUSED, BATCH_MATERIALIZED
    mats = _mixed()
    fused = batched_results(mats, modes=BATCH_FUSED)
    mat = batched_results(mats, modes=BATCH_MATERIALIZED)
    assert fused == mat
    assert mat == batched_results(mats)
    for pm, g in zip(mats[:10], mat[:10]):
        assert g == plain(pm), (pm.n, pm.degs)


@pytest.mark.parametrize("chunk_words", [None, 1, 3 * 400 * 121 * 101 + 5])
def test_materialized_chunks(chunk_words):
    """Materialized orders with the default chunk budget, one prime per
    chunk (budget 1 word) and three primes per chunk of the 20x20 job (a
    ragged last chunk): equal to the plain form."""
    from paper_2010_12117_gb300.binding import BATCH_MATERIALIZED
    rng = np.random.default_rng(31)
    big = synth.random_matrix(rng, 20, (6, 5), 0.6, -2000, 2000)  # 400 * 121 * 101 words per prime
    mats = [big, synth.random_matrix(rng, 3, (1,), 1.0, -5, 5), synth.random_matrix(rng, 16, (2,), 0.5, -9, 9),
            synth.random_matrix(rng, 20, (1, 1, 1), 0.4, -50, 50)]
    got = batched_results(mats, modes=BATCH_MATERIALIZED, chunk_words=chunk_words)
    for pm, g in zip(mats, got):
        assert g == plain(pm), (pm.n, pm.degs)


def test_full_grid_batch_equals_node_grid_batch():
    mats = _mixed()[:16]
    assert batched_results(mats, full_grid=True) == batched_results(mats)


def test_graph_replay_and_tuning_do_not_change_results():
    mats = _mixed()[:12]
    a = batched_results(mats)
    b = batched_results(mats, tune=True, graph=True, replays=3)
    assert a == b


def test_batched_workload_members_match_plain():
    mats = synth.batched(0, 256)[:40]
    got = batched_results(mats, tune=True, graph=True)
    for pm, g in zip(mats, got):
        assert g == plain(pm), pm.name
        cost = pm.n ** 3 * np.prod([pm.n * d + 1 for d in pm.degs])
        if cost < 1e6:
            assert g == bareiss.det_packed(pm.coeffs.tolist(), pm.degs), pm.name


def test_structured_and_singular_jobs():
    """Zero pivots (Sylvester, anti-diagonal), rank deficiency and zero
    matrices inside one batch."""
    k = 2
    rng = np.random.default_rng(9)
    mats = [synth.sylvester_16(5)]
    a = np.zeros((6, 6, 2), dtype=np.int64)
    for i in range(6):
        a[i, 5 - i] = [i + 1, 1]
    mats.append(synth.PolyMatrix(6, (1,), a))
    pm = synth.random_matrix(rng, 5, (2, 2), 0.8, -9, 10)
    M = P_.matrix_from_dense(pm.coeffs.tolist(), pm.degs)
    x = P_.var(0, k)
    M[3] = [P_.add(P_.mul(x, M[0][j]), M[2][j]) for j in range(5)]
    c = np.array([[P_.to_dense(M[i][j], (3, 2)) for j in range(5)] for i in range(5)], dtype=np.int64)
    mats.append(synth.PolyMatrix(5, (3, 2), c))
    mats.append(synth.PolyMatrix(7, (1, 1, 1), np.zeros((7, 7, 8), dtype=np.int64)))
    got = batched_results(mats)
    assert got[0] == bareiss.det_packed(mats[0].coeffs.tolist(), mats[0].degs)
    want = P_.const(-1, 1)
    for i in range(6):
        want = P_.mul(want, {(0,): i + 1, (1,): 1})
    assert P_.from_dense(got[1], (6,)) == want
    assert not any(got[2]) and not any(got[3])


def test_large_served_job_in_a_mix():
    """A 32x32 job over Z[x, y] with degree 6 (the served workload's large
    jobs) batched with small ones: equal to the plain path, certified."""
    rng = np.random.default_rng(1)
    big = synth.large_32x32_xy(rng)
    mats = [big] + synth.batched(7, 6)
    got = batched_results(mats)
    want_big = plain(big)
    assert got[0] == want_big
    from oracle import plan as oplan
    assert certificate.check(big.coeffs.tolist(), big.degs, got[0],
                             oplan.det_degree_bound(32, big.degs), trials=8)
    for pm, g in zip(mats[1:], got[1:]):
        assert g == plain(pm)


def test_last_variable_degree_limit():
    from paper_2010_12117_gb300.binding import Batch, PolydetError
    with pytest.raises(PolydetError):
        Batch([(4, (1, 8), 2)])


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_pipelined_end_to_end_runs_give_the_same_limbs(steps):
    """Upload, compute and download with each download overlapping the next
    run's compute: the results equal a plain run's."""
    from paper_2010_12117_gb300.runner import BatchedRunner
    mats = _mixed()[:14]
    want = batched_results(mats)
    st = torch.cuda.Stream()
    r = BatchedRunner(mats, tune=False, stream=st)
    r.capture(st)
    r.run_pipelined(steps, st)
    r.check_status(st)
    assert r.results() == want
    r.close()


def test_variable_reordering_round_trips():
    """Jobs whose variables the batched form reorders (lowest degree first for
    materialized orders, last for fused ones) come back in the caller's
    variable order: equal to the plain form, which keeps the order."""
    from paper_2010_12117_gb300.runner import variable_order
    rng = np.random.default_rng(77)
    mats = [synth.random_matrix(rng, 15, (3, 1, 2), 0.5, -99, 99), synth.random_matrix(rng, 6, (1, 3, 2), 0.7, -99, 99),
            synth.random_matrix(rng, 16, (2, 1), 0.6, -99, 99), synth.random_matrix(rng, 5, (1, 2), 1.0, -9, 9)]
    assert variable_order(15, (3, 1, 2)) == [1, 2, 0] and variable_order(6, (1, 3, 2)) == [1, 2, 0]
    got = batched_results(mats)
    for pm, g in zip(mats, got):
        assert g == plain(pm), (pm.n, pm.degs)


def test_batch_api_rejects_bad_settings():
    from paper_2010_12117_gb300.binding import BATCH_FUSED, Batch, PolydetError
    b = Batch([(5, (1, 2), 3), (16, (2,), 4)])
    try:
        with pytest.raises(PolydetError):
            b.set_mode(5, 7)
        with pytest.raises(PolydetError):
            b.set_mode(0, BATCH_FUSED)
        with pytest.raises(PolydetError):
            b.set_chunk_words(0)
        with pytest.raises(PolydetError):
            b.set_launch(16, 48)  # not a multiple of 32
        assert b.mode(5) == BATCH_FUSED and b.mode(16) == 1
        w0 = b.words["workspace"]
        b.set_chunk_words(1)  # one prime per chunk: the workspace shrinks or stays
        assert b.words["workspace"] <= w0
    finally:
        b.close()


def test_one_by_one_and_constant_jobs_in_both_modes():
    """Degenerate jobs: 1x1 matrices (the entry itself) and constant entries
    (degree 0 in every variable), fused and materialized."""
    from paper_2010_12117_gb300.binding import BATCH_FUSED, BATCH_MATERIALIZED
    rng = np.random.default_rng(3)
    mats = [synth.PolyMatrix(1, (3, 2), np.arange(12, dtype=np.int64).reshape(1, 1, 12) - 6),
            synth.random_matrix(rng, 4, (0,), 1.0, -9, 9), synth.random_matrix(rng, 15, (0, 0), 1.0, -9, 9),
            synth.random_matrix(rng, 3, (2, 0, 1), 0.9, -9, 9)]
    for mode in (BATCH_FUSED, BATCH_MATERIALIZED):
        got = batched_results(mats, modes=mode)
        assert got[0] == mats[0].coeffs[0, 0].tolist()
        for pm, g in zip(mats[1:], got[1:]):
            assert g == plain(pm), (mode, pm.n, pm.degs)


def test_withheld_bulk_copies_time_out_and_are_reported():
    """Failure detection without a fault: with the test hook on, the fused
    kernel's bounded wait for its staged rows runs out (about a second), the
    CTA sets the TIMEOUT bit of the status word and ends; with the hook off
    again the same batch gives the plain form's integers."""
    import time
    from paper_2010_12117_gb300.binding import BATCH_FUSED
    from paper_2010_12117_gb300.runner import BatchedRunner
    rng = np.random.default_rng(77)
    # last variable of degree 2 (L = 3, rows of n^2 x 4 words): every item's
    # rows start and end on 16 bytes, so every item takes the bulk copy
    mats = [synth.random_matrix(rng, n, (2, 3), 0.8, -50, 50) for n in (4, 6, 8)]
    want = [plain(pm) for pm in mats]
    st = torch.cuda.Stream()
    r = BatchedRunner(mats, tune=False, stream=st)
    r.set_modes(BATCH_FUSED)
    r.upload(st)
    r.batch.test_drop_copies(True)
    t0 = time.perf_counter()
    r.compute(st)
    st.synchronize()
    dt = time.perf_counter() - t0
    status = r.batch.sync_status(st)  # reads and clears every job's word
    assert status & 0x2, status
    assert 0.01 < dt < 60, dt  # the wait is bounded by time (1 s) or by a poll count
    r.batch.test_drop_copies(False)
    r.compute(st)
    r.download(st)
    st.synchronize()
    r.check_status(st)
    assert r.results() == want
    r.close()


def test_fused_staging_with_one_buffer_and_unaligned_rows():
    """Jobs whose last variable has degree 0 (one node per row, rows of n^2
    words): at n = 12, 13 two staging buffers do not fit in shared memory and
    the fused kernel runs with one; rows of odd n^2 words start off 16 bytes
    and are copied by the CTA, the others by bulk copies.  Same integers as
    the plain form."""
    from paper_2010_12117_gb300.binding import BATCH_FUSED
    rng = np.random.default_rng(91)
    mats = [synth.random_matrix(rng, 13, (2, 0), 0.7, -40, 40),
            synth.random_matrix(rng, 12, (0, 3), 0.7, -40, 40),
            synth.random_matrix(rng, 11, (1, 0), 0.9, -40, 40),
            synth.random_matrix(rng, 5, (0, 0, 2), 1.0, -40, 40)]
    got = batched_results(mats, modes=BATCH_FUSED)
    for pm, g in zip(mats, got):
        assert g == plain(pm), (pm.n, pm.degs)


@pytest.mark.parametrize("ctas", [1, 2])
def test_condensation_residency_cap_gives_the_same_results(ctas):
    """Capping the materialized orders' condensation CTAs per SM (reserved
    shared memory) changes only where the kernels run, not the integers."""
    from paper_2010_12117_gb300.binding import BATCH_MATERIALIZED
    from paper_2010_12117_gb300.runner import BatchedRunner
    mats = _mixed()[10:20]
    want = batched_results(mats, modes=BATCH_MATERIALIZED)
    st = torch.cuda.Stream()
    r = BatchedRunner(mats, tune=False, stream=st)
    r.set_modes(BATCH_MATERIALIZED)
    r.batch.set_condense_ctas(ctas)
    r.upload(st)
    r.compute(st)
    r.download(st)
    st.synchronize()
    r.check_status(st)
    assert r.results() == want
    r.close()
