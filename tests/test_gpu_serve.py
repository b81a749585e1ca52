"""Continuous batching: every request's result is the same served in a mix
as computed alone, waves overlap and the memory budget is respected."""
import numpy as np
import pytest

from helpers import ensure_lib
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _alone(pm):
    from paper_2010_12117_gb300.pipeline import determinant
    return determinant(pm.coeffs, pm.degs).coeffs


def test_served_results_equal_results_alone():
    from paper_2010_12117_gb300.serve import Server
    stream = synth.served_stream(3, 18, rate=400.0, large_frac=0.1)
    srv = Server(None, mem_budget=8e9, slots=2, wave_seconds=0.004, max_wave_jobs=6)
    rep = srv.run(stream)
    assert rep.jobs == len(stream)
    assert rep.waves > 1
    assert rep.p50_ms <= rep.p99_ms
    for d in rep.done:
        assert d.coeffs == _alone(stream[d.idx].job), stream[d.idx].job.name


def test_memory_budget_limits_what_is_in_flight():
    from paper_2010_12117_gb300.predictor import Predictor, shape_of
    from paper_2010_12117_gb300.serve import Server
    stream = synth.served_stream(4, 24, rate=2000.0, large_frac=0.0)
    pr = Predictor()
    mems = pr.predict([shape_of(a.job) for a in stream])[:, 1]
    budget = float(np.sort(mems)[-1] * 2.5)
    rep = Server(pr, mem_budget=budget, slots=3, wave_seconds=1.0).run(stream, keep_results=False)
    assert rep.jobs == len(stream)
    assert rep.peak_pred_mem <= budget
