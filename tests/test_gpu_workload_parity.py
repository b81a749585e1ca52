"""Every member of the 256-matrix batched workload (seed 0) through the
batched form, each checked by the oracle: bit-exact against O2 (integer
Bareiss after Kronecker packing) where its cost proxy n^3 prod(n d_v + 1) is
within the CPU budget, otherwise by the Schwartz-Zippel certificate O3 with
8 independent points mod 2^61 - 1.  The two counts are printed and, when the
run-output folder exists at the repository root, recorded there as JSON.
"""
import json
import multiprocessing
import os
import time

import numpy as np
import pytest

from helpers import ROOT, ensure_lib, oracle_check_member
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

O2_BUDGET = 5e6   # cost proxy up to which a member is checked bit-exactly (a few CPU seconds)
O3_TRIALS = 8


def test_every_member_of_the_batched_workload():
    ensure_lib()
    from paper_2010_12117_gb300.runner import BatchedRunner
    ctx = multiprocessing.get_context("spawn")
    workers = os.cpu_count() or 4
    with ctx.Pool(workers) as pool:
        mats = synth.batched(0, 256)
        st = torch.cuda.Stream()
        r = BatchedRunner(mats, tune=True, stream=st)
        r.upload(st)
        r.capture(st)
        r.compute(st)
        r.download(st)
        st.synchronize()
        r.check_status(st)
        got = r.results()
        r.close()
        cost = [pm.n ** 3 * float(np.prod([pm.n * d + 1 for d in pm.degs])) for pm in mats]
        tasks = [(pm.coeffs.tolist(), tuple(pm.degs), g, c <= O2_BUDGET)
                 for pm, g, c in zip(mats, got, cost)]
        # the largest first, so the pool's tail is short
        order = sorted(range(len(tasks)), key=lambda i: -cost[i])
        t0 = time.perf_counter()
        res = dict(zip(order, pool.map(oracle_check_member, [tasks[i] + (O3_TRIALS,) for i in order], chunksize=1)))
        wall = time.perf_counter() - t0
    bad = [(i, mats[i].n, mats[i].degs, res[i][0]) for i in range(len(mats)) if not res[i][1]]
    counts = {"exact_O2": sum(1 for v in res.values() if v[0] == "exact"),
              "certified_O3": sum(1 for v in res.values() if v[0] == "certified"),
              "o3_trials": O3_TRIALS, "o2_budget_cost_proxy": O2_BUDGET,
              "failed": len(bad), "members": len(mats), "oracle_wall_s": wall, "workers": workers,
              "oracle_cpu_s": sum(v[2] for v in res.values())}
    print("batched workload parity:", json.dumps(counts))
    out_dir = os.path.join(ROOT, "gpurun_out")
    if os.path.isdir(out_dir):
        with open(os.path.join(out_dir, "parity_batched256_seed0.json"), "w") as f:
            json.dump(counts, f)
    assert not bad, bad
    assert counts["exact_O2"] + counts["certified_O3"] == 256
