"""Stage-wise resume (Sec. 4.3): a run interrupted between primes, killed,
or left with a corrupt residue file resumes bit-exactly."""
import os
import signal
import subprocess
import sys

import numpy as np
import pytest

from helpers import ROOT, ensure_lib
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _run(pm, store=None, **kw):
    from paper_2010_12117_gb300.pipeline import determinant
    return determinant(pm.coeffs, pm.degs, store=store, **kw)


def test_interrupted_run_resumes_bit_exact(tmp_path):
    from paper_2010_12117_gb300.resume import ResidueStore
    pm = synth.sylvester_16(1)
    straight = _run(pm)
    store = ResidueStore(str(tmp_path / "r"))
    per_prime = 4 * (pm.n * pm.n * 128 + 128)
    with pytest.raises(InterruptedError):
        _run(pm, store=store, budget_bytes=3 * per_prime, stop_after_chunks=1)
    assert len(store.missing(straight.P, 97)) == straight.P - 3
    resumed = _run(pm, store=store, budget_bytes=3 * per_prime)
    assert resumed.coeffs == straight.coeffs
    assert store.missing(straight.P, 97) == []


def test_corrupt_or_truncated_residues_are_recomputed(tmp_path):
    from paper_2010_12117_gb300.resume import ResidueStore
    pm = synth.dense_4x4(2)
    straight = _run(pm)
    store = ResidueStore(str(tmp_path / "r"))
    _run(pm, store=store)
    C = 81
    f0 = os.path.join(store.path, "residues_p000.u32")
    data = bytearray(open(f0, "rb").read())
    data[10] ^= 0xFF
    open(f0, "wb").write(bytes(data))
    f1 = os.path.join(store.path, "residues_p001.u32")
    open(f1, "wb").write(open(f1, "rb").read()[:20])
    assert store.missing(straight.P, C) == [0, 1]
    again = _run(pm, store=store)
    assert again.coeffs == straight.coeffs
    assert store.missing(straight.P, C) == []


CHILD = r"""
import os, signal, sys
sys.path.insert(0, {root!r})
from paper_2010_12117_gb300 import synth
from paper_2010_12117_gb300.pipeline import determinant
from paper_2010_12117_gb300.resume import ResidueStore
import paper_2010_12117_gb300.resume as R
pm = synth.sylvester_16(2)
store = ResidueStore({path!r})
orig = R.ResidueStore.save
count = [0]
def save_then_die(self, q, r):
    orig(self, q, r)
    count[0] += 1
    if count[0] == 4:          # after the fourth prime is on disk, between launches
        os.kill(os.getpid(), signal.SIGKILL)
R.ResidueStore.save = save_then_die
determinant(pm.coeffs, pm.degs, store=store, budget_bytes=4 * (16 * 16 * 128 + 128))
"""


def test_killed_process_resumes(tmp_path):
    from paper_2010_12117_gb300.resume import ResidueStore
    path = str(tmp_path / "r")
    code = CHILD.format(root=ROOT, path=path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == -signal.SIGKILL, r.stderr
    pm = synth.sylvester_16(2)
    straight = _run(pm)
    store = ResidueStore(path)
    assert len(store.missing(straight.P, 97)) == straight.P - 4
    assert _run(pm, store=store).coeffs == straight.coeffs
