#!/usr/bin/env python3
"""Throughput of exact polynomial-matrix determinants on GB300.

Workload (one step): the batched workload of the method - 256 matrices over
Z[x1..xk], n ~ U[4, 24], k ~ U{1, 2, 3}, entry degree d_v ~ U[1, 4],
monomial density ~ U[0.3, 1.0], int16 coefficients, seeded - each taken to
its exact determinant (every prime: evaluation, condensation, interpolation;
then Garner CRT).  Inputs are resident in HBM when the timed region starts;
L2 is flushed (256 MiB write) before every timed step, outside the timing.

One JSON line on stdout (rank 0).  ``--impl reference`` times the CPU oracle
(plain Python Bareiss after Kronecker packing) on a bounded sample instead.
Under torchrun each rank runs its own batch (seed + rank): weak scaling with
no collective on the data path; only the timing barrier and a max over ranks.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("exact poly determinants/sec and mod-p n×n dets/sec; IMAD % and HBM GB/s of peak")
# DRAM traffic of condense_kernel measured by ncu (read + write over the
# algorithmic bytes 4 n^2 + 4 per determinant, from one capture of a single
# 24 x 24 launch, with the IMAD pipe's active fraction from the same
# capture), valid only for the code it was taken on: digests of the
# kernel's sources with comments and blank space removed; the bench reports
# traffic null once they change.
CONDENSE_TRAFFIC = {"ratio": 1.0133, "fmaheavy_active": 0.716,
                    "sources": {"paper_2010_12117_gb300/csrc/condense.cuh": "b0dcc202ebcb755b",
                                "paper_2010_12117_gb300/csrc/modarith.cuh": "b36f048e62c9ded4",
                                "paper_2010_12117_gb300/csrc/teams.cuh": "2b54f7c70ebf5672"}}


def _code_digest(path: str) -> str:
    import hashlib
    import re
    with open(os.path.join(ROOT, path)) as f:
        s = f.read()
    s = re.sub(r"/\*.*?\*/", "", s, flags=re.S)
    s = re.sub(r"//[^\n]*", "", s)
    s = re.sub(r"\s+", "", s)
    return hashlib.sha256(s.encode()).hexdigest()[:16]


def _sources_match(sources: dict) -> bool:
    return all(_code_digest(path) == h for path, h in sources.items())


def _traffic_ratio():
    return CONDENSE_TRAFFIC["ratio"] if _sources_match(CONDENSE_TRAFFIC["sources"]) else None


# Active fraction of the FMA-heavy (IMAD) pipe in crt_kernel_p<11> on 2^24
# coefficients, from one ncu capture, valid for the sources it was taken on.
CRT_PIPE = {"fmaheavy_active": {11: 0.843},
            "sources": {"paper_2010_12117_gb300/csrc/crt.cu": "b7f51ef1688995fc",
                        "paper_2010_12117_gb300/csrc/modarith.cuh": "b36f048e62c9ded4"}}
# The same for the x_1 pass (coltx_direct_kernel<4, 2>) of the node-grid
# evaluation (37^3 nodes, 20 primes), the pass that moves its bytes.
EVAL_PIPE = {"fmaheavy_active": 0.779,
             "sources": {"paper_2010_12117_gb300/csrc/ntt_direct.cuh": "cca188a993a99705",
                         "paper_2010_12117_gb300/csrc/modarith.cuh": "b36f048e62c9ded4"}}


WORKLOAD = ("batched: 256 matrices, n~U[4,24], k~U{1,2,3}, d_v~U[1,4], density~U[0.3,1.0], "
            "int16 coefficients, seeded")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-kernels", action="store_true")
    ap.add_argument("--no-structured", action="store_true")
    ap.add_argument("--served-jobs", type=int, default=2000)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (weak scaling, no data-path collective)
# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    """Units processed by all ranks (each rank runs its own batch)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv",
                                       "-lms", "200", "-i", str(self.gpu)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self) -> dict:
        self.f.flush()
        self.f.seek(0)
        rows = list(csv.reader(io.StringIO(self.f.read())))
        os.unlink(self.f.name)
        if len(rows) < 2:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        head = [h.strip() for h in rows[0]]
        data = [[c.strip() for c in r] for r in rows[1:] if len(r) == len(head)]

        def col(name):
            i = next(i for i, h in enumerate(head) if h.startswith(name))
            return [r[i] for r in data]

        def num(s):
            try:
                return float(s.split()[0])
            except (ValueError, IndexError):
                return None

        sm = [v for v in map(num, col("clocks.current.sm")) if v is not None]
        mx = [v for v in map(num, col("clocks.max.sm")) if v is not None]
        reasons = []
        for name, key in (("hw_slowdown", "clocks_event_reasons.hw_slowdown"),
                          ("hw_thermal_slowdown", "clocks_event_reasons.hw_thermal_slowdown"),
                          ("sw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown"),
                          ("sw_power_cap", "clocks_event_reasons.sw_power_cap")):
            try:
                if any(v.lower() == "active" for v in col(key)):
                    reasons.append(name)
            except StopIteration:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_cost(pm) -> float:
    """Rough O2 cost proxy: n^3 big-integer products of the packed det size."""
    import numpy as np
    positions = float(np.prod([pm.n * d + 1 for d in pm.degs]))
    return pm.n ** 3 * positions


def _oracle_det(item):
    """One member through the oracle (runs in a pool worker): (index, det)."""
    from oracle import bareiss
    idx, coeffs, degs = item
    return idx, bareiss.det_packed(coeffs, degs)


class OraclePool:
    """The members of the seeded batch whose cost proxy is at most ``cap``, in
    seed order, and a spawn-started pool of processes over the host's cores
    that runs them through the oracle one member per task (start-up and
    imports happen here, outside any timing)."""

    def __init__(self, mats, cap: float = 2e6, workers: int = 0):
        import multiprocessing
        self.eligible = [(i, pm.coeffs.tolist(), tuple(pm.degs)) for i, pm in enumerate(mats)
                         if oracle_cost(pm) <= cap]
        self.skipped = len(mats) - len(self.eligible)
        self.workers = workers or os.cpu_count() or 1
        self.pool = multiprocessing.get_context("spawn").Pool(self.workers)
        self.pool.map(_oracle_det, self.eligible[:self.workers])
        self.next = 0

    def window(self, seconds: float):
        """Keep every worker busy with the next member (cycling through the
        eligible ones) for ``seconds`` of wall time.  Returns the completion
        times (seconds from the start) of the members finished inside the
        window; members still running when it ends are not counted (close()
        ends them), so the window's length bounds the run.  ``self.results``
        maps each finished member's index to the oracle's determinant."""
        self.results = {}
        import queue
        done_q = queue.SimpleQueue()
        t0 = time.perf_counter()

        def submit():
            item = self.eligible[self.next % len(self.eligible)]
            self.next += 1
            self.pool.apply_async(_oracle_det, (item,), callback=done_q.put, error_callback=done_q.put)

        for _ in range(self.workers):
            submit()
        times = []
        while True:
            left = seconds - (time.perf_counter() - t0)
            if left <= 0:
                break
            try:
                r = done_q.get(timeout=left)
            except queue.Empty:
                break
            if isinstance(r, BaseException):
                raise r
            t = time.perf_counter() - t0
            if t > seconds:
                break
            times.append(t)
            self.results[r[0]] = r[1]
            submit()
        return times

    def close(self):
        self.pool.terminate()
        self.pool.join()


def run_reference(args, world, rank):
    from paper_2010_12117_gb300 import synth
    if rank != 0:
        return
    mats = synth.batched(args.seed, args.count)
    # the steps are consecutive slices of one window of at most two minutes
    el = min(args.steps * max(2.0, args.cpu_seconds / 2), 120.0)
    per_step = el / args.steps
    pool = OraclePool(mats)
    try:
        done = len(pool.window(el))
    finally:
        pool.close()
    workers = pool.workers
    value = done / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "exact dets/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "python int (exact)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "seed": args.seed, "sample": "cost-capped members in seed order"},
        "cpu_baseline": {"value": value, "unit": "exact dets/s", "cores": workers, "kind": "oracle",
                         "sample": f"{done} members finished in {args.steps} steps of {per_step:.1f} s, one per "
                                   f"process on {workers} cores: members of the seeded batch in order "
                                   "whose n^3*prod(n d_v+1) <= 2e6 (small ones; larger ones are out of "
                                   "reach of the Python oracle)"},
        "e2e": {"value": value, "unit": "exact dets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(_plain(line)), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def _timed_steps(runner, st, flush, steps, stage_timer):
    """``steps`` timed passes, L2 flushed before each outside the events;
    stage events between the stage graphs.  Returns per-rank total ms."""
    import torch
    marks = []
    for _ in range(steps):
        with torch.cuda.stream(st):
            flush.fill_(2)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(st)
        runner.compute(st, stage_timer)
        e.record(st)
        marks.append((s, e))
    torch.cuda.synchronize()
    return sum(s.elapsed_time(e) for s, e in marks)


def served_leg(args, mats, batched_value, st):
    """The served workload: a seeded Poisson stream of the batched
    distribution plus 5 % 32x32 jobs over Z[x, y] (degree 6), continuous
    batching with admission by predicted memory.  First the server's
    capacity (the same jobs all waiting at t = 0, MLP admission, an ample
    budget), then a sweep of arrival rates at 0.5x, 1x and 2x that capacity
    under a memory budget that binds (60 % of the device memory the waves
    actually held at peak at capacity), once per admission policy: the MLP trained on the method's
    own timings, the analytic bound calibrated by its median ratio to the
    measurements, and the raw bound.  Each run reports p50/p99 latency,
    dets/s and the device memory its waves actually held at peak against the
    budget."""
    import numpy as np
    import torch
    from paper_2010_12117_gb300 import synth
    from paper_2010_12117_gb300.predictor import Predictor
    from paper_2010_12117_gb300.serve import Server, calibrate
    rng = np.random.default_rng(args.seed + 1000)
    cal = synth.batched(args.seed + 100, 60) + [synth.large_32x32_xy(rng) for _ in range(4)]
    t0 = time.perf_counter()
    X, Y, Bd = calibrate(cal, st)
    pr = Predictor(seed=args.seed)
    pr.fit(X, Y, Bd, steps=2000)
    train_s = time.perf_counter() - t0
    calibrated = Predictor(seed=args.seed)
    calibrated.ratio = pr.ratio.copy()  # untrained: the bound times the measured median ratio
    policies = (("mlp", pr), ("calibrated_bound", calibrated), ("raw_bound", Predictor(seed=args.seed)))
    base_stream = synth.served_stream(args.seed, args.served_jobs, rate=1.0)
    backlog = [synth.Arrival(0.0, a.job) for a in base_stream]

    def run(pred, arrivals, budget):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        rep = Server(pred, mem_budget=budget, slots=3, wave_seconds=0.02).run(arrivals, keep_results=False)
        torch.cuda.synchronize()
        actual = float(torch.cuda.max_memory_allocated() - base)
        return dict(rep.summary(), budget_bytes=float(budget), actual_peak_bytes=actual,
                    over_budget=bool(actual > float(budget)))

    run(pr, backlog[:40], 200e9)  # warm: plan tables, batch resources, allocator
    caps = [run(pr, backlog, 200e9) for _ in range(2)]  # two runs: the capacity varies by +-5 %
    cap = max(caps, key=lambda c: c["exact_dets_per_s"])
    cap["runs_exact_dets_per_s"] = [c["exact_dets_per_s"] for c in caps]
    capacity = cap["exact_dets_per_s"]
    # 60 % of the device memory the waves held at peak with nothing binding
    # (above what the largest job needs alone): an admission policy that
    # under-predicts memory overruns it
    budget = 0.6 * float(cap["actual_peak_bytes"])
    out = {"jobs": args.served_jobs, "calibration_jobs": len(cal), "calibrate_and_train_s": train_s,
           "slots": 3, "capacity": cap, "binding_budget_bytes": budget, "rates": {}}
    for frac in (0.5, 1.0, 2.0):
        rate = frac * capacity
        stream = synth.served_stream(args.seed, args.served_jobs, rate=rate)
        out["rates"][f"{frac}x"] = {"rate_jobs_per_s": rate}
        for name, p in policies:
            out["rates"][f"{frac}x"][name] = run(p, stream, budget)
    # the plain per-matrix form over the same jobs (one pass, CUDA events)
    from paper_2010_12117_gb300.runner import PlainRunner
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    plain = PlainRunner([a.job for a in base_stream])  # plans, buffers, upload, run, download
    plain.upload(st)
    plain.compute(st)
    plain.download(st)
    st.synchronize()
    wall = time.perf_counter() - w0
    s_ev = torch.cuda.Event(enable_timing=True)
    e_ev = torch.cuda.Event(enable_timing=True)
    s_ev.record(st)
    plain.compute(st)
    e_ev.record(st)
    e_ev.synchronize()
    ms = s_ev.elapsed_time(e_ev)
    plain.close()
    out["plain_same_jobs"] = {"wall_s": wall, "exact_dets_per_s": len(base_stream) / wall,
                              "device_ms": ms, "device_exact_dets_per_s": len(base_stream) / (ms * 1e-3),
                              "note": "wall: plans, buffers, upload, one pass, download (like the "
                                      "server's waves); device: one pass with inputs resident"}
    return out


def kernel_leg(st, hbm_peak, mats):
    """Stages alone on inputs larger than L2 (the 12x12 trivariate workload):
    evaluation on the node grid (37^3 nodes, 20 primes: 583 MB written) and on
    the paper's full grid (64^3 nodes, 5 primes: 755 MB), interpolation on
    both grids (inverse NTT on the full grid; the node grid's coset-structured
    solve), and the CRT on 2^24 coefficients with 6 and 11 primes."""
    import numpy as np
    import torch
    from paper_2010_12117_gb300 import synth
    from paper_2010_12117_gb300.binding import Plan

    def timed(fn, reps=5):
        fn()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(st)
        for _ in range(reps):
            fn()
        e.record(st)
        e.synchronize()
        return s.elapsed_time(e) / reps

    def hbm(ms, byts):
        return {"ms": ms, "GBps": byts / ms / 1e6, "frac": byts / ms / 1e6 / hbm_peak,
                "algorithmic_bytes": byts, "bound": "hbm"}

    out = {}
    pm = synth.sparse_12x12_xyz(0)
    c = torch.from_numpy(pm.coeffs.astype(np.int32).reshape(-1)).cuda()
    n2 = pm.n * pm.n
    for name, P, full in (("node_grid_37^3_P20", 20, False), ("full_grid_64^3_P5", 5, True)):
        pl = Plan(pm.n, pm.degs, P, full_grid=full)
        ev = torch.empty(P * n2 * pl.G, dtype=torch.int32, device="cuda")
        ws = pl.workspace(P)
        ms = timed(lambda: pl.eval(c, 0, P, ev, ws, st))
        out[f"eval_{name}"] = hbm(ms, 4.0 * P * n2 * (pl.E + pl.G))
        if not full and _sources_match(EVAL_PIPE["sources"]):
            # its x_1 pass keeps the integer multiply pipe this busy (ncu)
            out[f"eval_{name}"]["x1_pass_imad_pipe_active_ncu"] = EVAL_PIPE["fmaheavy_active"]
        dv = torch.empty(P * pl.G, dtype=torch.int32, device="cuda")
        pl.condense(ev, 0, P, dv, st)
        del ev
        rs = torch.empty(P * pl.C, dtype=torch.int32, device="cuda")
        ms = timed(lambda: pl.interp(dv, 0, P, rs, ws, st))
        if full:
            out[f"interp_{name}"] = hbm(ms, 4.0 * P * (pl.G + pl.C))
        else:
            # work of a dense inverse Vandermonde per line (M_v^2 products); the
            # coset-structured solve does about M_v^2 / L of them
            macs = float(P) * sum(pl.M[v] * math.prod(pl.M[:v]) * math.prod(x + 1 for x in pl.D[v:])
                                  for v in range(pl.k))
            out[f"interp_{name}"] = {"ms": ms, "dense_equiv_Gmac_per_s": macs / ms / 1e6, "bound": "alu",
                                     "dense_equiv_macs": macs, "GBps": 4.0 * P * (pl.G + pl.C) / ms / 1e6}
        pl.close()
        del dv, rs, ws
        torch.cuda.empty_cache()
    for P in (6, 11):
        pc = Plan(1, (4095, 4095), P)  # C = 4096^2 = 2^24 coefficients
        C = pc.C
        res = torch.randint(0, 2 ** 30, (P * C,), dtype=torch.int32, device="cuda")
        limbs = torch.empty(C * pc.W, dtype=torch.int32, device="cuda")
        ms = timed(lambda: pc.crt(res, limbs, st))
        byts = 4.0 * C * (P + pc.W)
        W = pc.W
        # the integer side: Garner P (P - 1) / 2 mulmods and P W limb products
        mulmods = float(C) * (P * (P - 1) / 2 + P * W)
        out[f"crt_2^24_P{P}"] = dict(hbm(ms, byts), W=W, mulmods_per_s=mulmods / (ms * 1e-3))
        pipe = CRT_PIPE["fmaheavy_active"].get(P)
        if pipe is not None and _sources_match(CRT_PIPE["sources"]):
            # the integer multiply pipe, not memory, bounds it (ncu)
            out[f"crt_2^24_P{P}"].update(bound="imad", imad_pipe_active_ncu=pipe)
        pc.close()
        del res, limbs
    torch.cuda.empty_cache()
    out["eval_batched_workload"] = eval_totals(mats, st, hbm_peak)
    torch.cuda.empty_cache()
    return out


def eval_totals(mats, st, hbm_peak):
    """The evaluation (every NTT pass) of every job of the batched workload,
    one job after another through the per-matrix API, in the variable order
    the batched form uses: aggregate algorithmic bytes (int32 coefficients in,
    evaluated matrices out) over the sum of the launches' event times."""
    import numpy as np
    import torch
    from paper_2010_12117_gb300.binding import Plan
    from paper_2010_12117_gb300.pipeline import prime_count
    from paper_2010_12117_gb300.runner import permute_coeffs, variable_order
    budget = 1 << 29  # words of evaluated matrices per launch group
    plans = []
    most, ws_most = budget, 1
    for pm in mats:
        order = variable_order(pm.n, pm.degs)
        degs = tuple(pm.degs[v] for v in order)
        pl = Plan(pm.n, degs, prime_count(pm.coeffs))
        c = torch.from_numpy(np.ascontiguousarray(permute_coeffs(pm.coeffs, pm.degs, order),
                                                  dtype=np.int32).reshape(-1)).cuda()
        per = pm.n * pm.n * pl.G
        cp = max(1, min(pl.P, budget // per))
        most = max(most, cp * per)
        ws_most = max(ws_most, cp * pl.eval_ws_words)
        plans.append((pm, pl, c, cp))
    buf = torch.empty(most, dtype=torch.int32, device="cuda")
    wsb = torch.empty(ws_most, dtype=torch.int32, device="cuda")
    ms_total, byts = 0.0, 0.0
    for rep in range(2):  # the first pass warms up
        evs = []
        for pm, pl, c, cp in plans:
            for lo in range(0, pl.P, cp):
                hi = min(pl.P, lo + cp)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                pl.eval(c, lo, hi, buf, wsb, st)
                b.record(st)
                evs.append((a, b, 4.0 * (hi - lo) * pm.n * pm.n * (pl.E + pl.G)))
        st.synchronize()
        if rep:
            ms_total = sum(a.elapsed_time(b) for a, b, _ in evs)
            byts = sum(x for _, _, x in evs)
    for _, pl, _, _ in plans:
        pl.close()
    return {"ms": ms_total, "GBps": byts / ms_total / 1e6, "frac": byts / ms_total / 1e6 / hbm_peak,
            "algorithmic_bytes": byts, "bound": "hbm", "launch_groups": len(evs)}


def structured_leg(st, hbm_peak, derived_upd):
    """Sec. 3.1's large-degree case and Sec. 5/6's repeated entries.

    (1) The 15 x 15 Sylvester matrix over Z[x1..x4] with determinant degrees
    (298, 171, 119, 45): 2.8e8 nodes per prime, evaluation + condensation
    streamed slab by slab through a fixed workspace (the lowest-degree
    variable first: its nodes are the slabs), then interpolation and CRT;
    once with the entry map (17 distinct entries + the zero one of 225) in a
    24 GB workspace, once with all 225 entries in 64 GB (one prime's
    evaluated matrices would take 255 GB).  (2) The 16 x 16 Sylvester
    workload's evaluation with and without the entry map (18 distinct of
    256 entries)."""
    import numpy as np
    import torch
    from paper_2010_12117_gb300 import synth
    from paper_2010_12117_gb300.binding import Plan, det_degree_bound, entry_degrees, unique_entries
    from paper_2010_12117_gb300.pipeline import permute_coeffs, prime_count
    from paper_2010_12117_gb300.runner import condense_updates

    def ev_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    out = {}
    pm = synth.sylvester_15_four_vars(0)
    order = sorted(range(pm.nvars), key=lambda v: (pm.degs[v], v))
    cp = permute_coeffs(pm.coeffs, pm.degs, order)
    dp = tuple(pm.degs[v] for v in order)
    D = det_degree_bound(entry_degrees(cp, dp), len(dp))
    P = prime_count(pm.coeffs)
    m, U, uniq = unique_entries(cp)
    for name, use_map, budget in (("entry_map_24GB", True, 24 << 30), ("all_entries_64GB", False, 64 << 30)):
        pl = Plan(pm.n, dp, P, det_degs=D)
        rows = np.ascontiguousarray(cp, dtype=np.int32).reshape(pm.n * pm.n, -1)
        if use_map:
            pl.set_entry_map(m, U)
            rows = uniq
        c = torch.from_numpy(np.ascontiguousarray(rows, dtype=np.int32).reshape(-1)).cuda()
        ws_words = max(pl.stream_ws_words(1), pl.interp_ws_words, min(pl.stream_ws_words(pl.M[0]), budget // 4))
        ws = torch.empty(ws_words, dtype=torch.int32, device="cuda")
        detv = torch.empty(pl.G, dtype=torch.int32, device="cuda")
        res = torch.empty(P * pl.C, dtype=torch.int32, device="cuda")
        limbs = torch.empty(pl.C * pl.W, dtype=torch.int32, device="cuda")
        pl.eval_condense(c, 0, 1, detv, ws, st)  # warm: module load, attributes
        st.synchronize()
        marks = {"eval_condense": [], "interp": [], "crt": []}
        for q in range(P):
            a, b = ev_pair()
            a.record(st)
            pl.eval_condense(c, q, q + 1, detv, ws, st)
            b.record(st)
            marks["eval_condense"].append((a, b))
            a, b = ev_pair()
            a.record(st)
            pl.interp(detv, q, q + 1, res[q * pl.C:(q + 1) * pl.C], ws, st)
            b.record(st)
            marks["interp"].append((a, b))
        a, b = ev_pair()
        a.record(st)
        pl.crt(res, limbs, st)
        b.record(st)
        marks["crt"].append((a, b))
        st.synchronize()
        status = pl.sync_status(st)
        ms = {k: sum(x.elapsed_time(y) for x, y in v) for k, v in marks.items()}
        upd = float(P) * pl.G * condense_updates(pm.n)
        row_words = pl.entries * -(-(pl.G // pl.M[0]) // 32) * 32
        slab_rows = min(pl.M[0], max(1, (ws_words - pl.items * (pl.G // pl.M[0]) * (pl.d[0] + 1)) // row_words))
        out[name] = {"n": pm.n, "det_degrees_in_order": [int(x) for x in pl.D], "variable_order": order,
                     "P": P, "G": pl.G, "C": pl.C, "W": pl.W, "entries_per_prime": pl.entries,
                     "evaluated_bytes_per_prime": 4.0 * pl.entries * pl.G,
                     "workspace_bytes": 4.0 * ws_words, "approx_slab_rows_of_x1": int(slab_rows),
                     "ms": ms, "total_ms": sum(ms.values()), "status": status,
                     "modp_dets_per_s": P * pl.G / (ms["eval_condense"] * 1e-3),
                     "eval_condense_Gupdate_s": upd / (ms["eval_condense"] * 1e-3) / 1e9,
                     "eval_condense_alu_frac": upd / (ms["eval_condense"] * 1e-3) / derived_upd,
                     "bound": "alu"}
        pl.close()
        del c, ws, detv, res, limbs
        torch.cuda.empty_cache()
    # the 16 x 16 Sylvester workload: evaluation with and without the map
    pm = synth.sylvester_16(0)
    P = prime_count(pm.coeffs)
    m, U, uniq = unique_entries(pm.coeffs)
    res16 = {}
    for name, use_map in (("all_entries", False), ("entry_map", True)):
        pl = Plan(pm.n, pm.degs, P)
        rows = np.ascontiguousarray(pm.coeffs, dtype=np.int32).reshape(pm.n * pm.n, -1)
        if use_map:
            pl.set_entry_map(m, U)
            rows = uniq
        c = torch.from_numpy(np.ascontiguousarray(rows, dtype=np.int32).reshape(-1)).cuda()
        ev = torch.empty(P * pl.entries * pl.G, dtype=torch.int32, device="cuda")
        dv = torch.empty(P * pl.G, dtype=torch.int32, device="cuda")
        wsb = pl.workspace(P)
        pl.eval(c, 0, P, ev, wsb, st)
        reps = 200
        a, b = ev_pair()
        a.record(st)
        for _ in range(reps):
            pl.eval(c, 0, P, ev, wsb, st)
        b.record(st)
        a2, b2 = ev_pair()
        a2.record(st)
        for _ in range(reps):
            pl.condense(ev, 0, P, dv, st)
        b2.record(st)
        st.synchronize()
        res16[name] = {"entries_per_prime": pl.entries, "evals_bytes": 4.0 * P * pl.entries * pl.G,
                       "eval_us": 1e3 * a.elapsed_time(b) / reps, "condense_us": 1e3 * a2.elapsed_time(b2) / reps}
        pl.close()
    res16["eval_bytes_ratio"] = res16["all_entries"]["evals_bytes"] / res16["entry_map"]["evals_bytes"]
    res16["eval_time_ratio"] = res16["all_entries"]["eval_us"] / res16["entry_map"]["eval_us"]
    out["sylvester_16x16_eval"] = res16
    # early termination on a determinant far below its coefficient bound
    # (wall clock of the public call: one prime at a time, a check per prime)
    from paper_2010_12117_gb300.binding import limbs_to_ints
    from paper_2010_12117_gb300.pipeline import determinant
    pm = synth.small_det_matrix(np.random.default_rng(7), 24, (3, 3, 3), (1, 1, 1), mixes=24)
    determinant(pm.coeffs, pm.degs, early_stop=True, as_ints=False)  # warm: plans, kernels
    et, vals = {}, {}
    for name, es in (("full_count", False), ("early_stop", True)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = determinant(pm.coeffs, pm.degs, early_stop=es, as_ints=False)
        torch.cuda.synchronize()
        et[name] = {"ms": 1e3 * (time.perf_counter() - t), "primes": r.P, "bound_primes": r.primes_bound,
                    "modp_dets": r.P * int(np.prod([x + 1 for x in r.D]))}
        vals[name] = limbs_to_ints(r.limbs, r.W)
    et["workload"] = "24x24 over Z[x,y,z], degree 3, determinant of degree 24 per variable with coefficients " \
                     "far below the Hadamard bound (small_det_matrix seed 7)"
    et["identical_output"] = vals["full_count"] == vals["early_stop"]
    et["speedup"] = et["full_count"]["ms"] / et["early_stop"]["ms"]
    out["early_termination"] = et
    return out


def run_ours(args, world, rank, local):
    import torch
    from paper_2010_12117_gb300 import synth
    from paper_2010_12117_gb300.binding import condense_steps, probe_int_peaks
    from paper_2010_12117_gb300.runner import BatchedRunner, PlainRunner, StageTimer

    torch.cuda.set_device(local)
    dev_props = torch.cuda.get_device_properties(local)
    mats = synth.batched(args.seed + rank, args.count)
    st = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # batched form: tuned, captured once in a CUDA graph (stage events inside)
    runner = BatchedRunner(mats, tune=True, stream=st)
    runner.upload(st)
    runner.capture(st)
    for _ in range(args.warmup):
        with torch.cuda.stream(st):
            flush.fill_(1)
        runner.compute(st)
    torch.cuda.synchronize()
    runner.check_status(st)

    barrier(world)
    torch.cuda.synchronize()
    timer = StageTimer()
    with ClockSampler(local) as clk:
        my_ms = _timed_steps(runner, st, flush, args.steps, timer)
    stage_ms = timer.ms()
    barrier(world)
    total_ms = max_over_ranks(my_ms, world)
    clocks = clk.summary()
    runner.check_status(st)
    exact_per_step = len(mats)
    modp_per_step = runner.modp_dets()
    exact_all = sum_over_ranks(float(exact_per_step), world)
    modp_all = sum_over_ranks(float(modp_per_step), world)
    value = exact_all * args.steps / (total_ms * 1e-3)
    modp_value = modp_all * args.steps / (total_ms * 1e-3)

    # end to end through the public runner: every step uploads its inputs from
    # pinned host memory, computes, and downloads its limbs to pinned host
    # memory; a step's download overlaps the next step's compute
    cs = torch.cuda.Stream()
    runner.run_pipelined(args.warmup, st, cs)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    runner.run_pipelined(args.steps, st, cs)
    e2e_ms = 1e3 * (time.perf_counter() - t0)
    runner.check_status(st)  # the pipelined runs' status word (raises when set)
    e2e_total = max_over_ranks(e2e_ms, world)
    e2e_value = exact_all * args.steps / (e2e_total * 1e-3)
    batched_results = runner.results()
    launches = runner.kernel_launches() * args.steps
    h2d, d2h = runner.h2d_bytes, runner.d2h_bytes
    tuning = {str(n): ("materialized" if v.get("mode") else f"fused/{v.get('threads')}")
              for n, v in runner.tuning.items()}
    work = dict(timer.work)
    runner.close()
    del runner
    torch.cuda.empty_cache()

    # the plain per-matrix GPU form on the same batch (comparison; identical output)
    plain = PlainRunner(mats)
    plain.upload(st)
    plain.compute(st)
    torch.cuda.synchronize()
    ps = torch.cuda.Event(enable_timing=True)
    pe = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        flush.fill_(3)
    ps.record(st)
    plain.compute(st)
    pe.record(st)
    plain.download(st)
    torch.cuda.synchronize()
    plain_ms = ps.elapsed_time(pe)
    plain_max = max_over_ranks(plain_ms, world)
    same = plain.results() == batched_results
    # one more plain pass with an event pair around every launch: the
    # condensation kernel's own launch durations (graph replays of the
    # batched form cannot carry events between their kernels)
    ptimer = StageTimer()
    with torch.cuda.stream(st):
        flush.fill_(4)
    plain.compute(st, ptimer)
    torch.cuda.synchronize()
    plain.check_status(st)
    plain_stage_ms = ptimer.ms()
    # algorithmic bytes of the condensation launches: 4 n^2 + 4 per determinant
    cond_bytes = sum(float(pl.P * pl.G) * (4 * pm.n * pm.n + 4) for pm, pl in zip(plain.mats, plain.plans))
    bytes_by_order = {}
    for pm, pl in zip(plain.mats, plain.plans):
        bytes_by_order[pm.n] = bytes_by_order.get(pm.n, 0.0) + float(pl.P * pl.G) * (4 * pm.n * pm.n + 4)
    plain.close()
    del plain

    # roofline of the dominant kernel
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    imad_s, upd1_s, pair_s, triple_s = probe_int_peaks(st)
    sms = dev_props.multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    lanes = sms * 64 * sm_mhz * 1e6  # IMAD lanes per second (64 per SM per clock)
    # The condensation kernel of order n takes its elimination steps two or
    # three at a time (condense_steps).  One element update of a step pair
    # (two algorithmic updates) issues three 32x32->64-bit multiply-adds and
    # the REDC's IMAD and IMAD.HI; the pipe costs ncu measures on the probes
    # (a wide multiply-add or an IMAD.HI holds the FMA-heavy pipe two slots,
    # an IMAD one) make that 9 slots, 4.5 per update; one of a step triple
    # (three updates) four multiply-adds and the same two: 11 slots, 11/3 per
    # update.  The probes run both element updates in registers.
    slots = {2: 4.5, 3: 11.0 / 3.0}
    probe_upd = {2: 2.0 * pair_s, 3: 3.0 * triple_s}
    step_of = {n_: condense_steps(n_) for n_ in range(1, 33)}

    def model_peak(n_):
        return lanes / slots[step_of[n_]]
    single_step_upd = lanes / 6.0  # the single-step kernel's model (6 slots), kept for comparison
    peak_src = (f"derived: {sms} SMs x 64 IMAD/clk x {sm_mhz:.0f} MHz / IMAD slots per update "
                "of each order's pass (4.5 for a step pair, 11/3 for a step triple), weighted by "
                "each order's updates")
    # per order: the update rate against its integer-pipe peak, the byte rate
    # against HBM, and the time either bound alone allows; the sum of those
    # times over the sum of the measured ones is the kernel's fraction of its
    # launch-by-launch roofline (small orders read 4 n^2 bytes for only
    # (n-1) n (2n-1) / 6 updates and are HBM-bound)
    by_order, t_bound, t_meas = {}, 0.0, 0.0
    t_model = t_probe = upd_all = 0.0
    for n_, (ms_, upd) in sorted(ptimer.tag_ms("condense").items()):
        byt = bytes_by_order[n_]
        pk = model_peak(n_)
        tb = max(upd / pk, byt / (hbm_peak * 1e9))
        t_bound += tb
        t_meas += ms_ * 1e-3
        t_model += upd / pk
        t_probe += upd / probe_upd[step_of[n_]]
        upd_all += upd
        by_order[str(n_)] = {"ms": ms_, "steps_per_pass": step_of[n_], "Gupdate_s": upd / (ms_ * 1e-3) / 1e9,
                             "alu_frac": upd / (ms_ * 1e-3) / pk,
                             "alu_frac_of_probe": upd / (ms_ * 1e-3) / probe_upd[step_of[n_]],
                             "alu_frac_of_single_step_peak": upd / (ms_ * 1e-3) / single_step_upd,
                             "hbm_frac": byt / (ms_ * 1e-3) / (hbm_peak * 1e9),
                             "bound": "alu" if upd / pk >= byt / (hbm_peak * 1e9) else "hbm"}
    # the batch's work-weighted ceilings (the batched form condenses the same
    # determinants of every order)
    derived_upd = upd_all / t_model if t_model else lanes / 4.5
    upd_s = upd_all / t_probe if t_probe else 2.0 * pair_s

    def roofs_of(stage_ms, work):
        roofs = {}
        for name, ms in stage_ms.items():
            w = work.get(name, 0.0)  # summed over the timed passes
            ach = w / (ms * 1e-3) / 1e9
            if name == "condense":
                roofs[name] = {"bound": "alu", "achieved": ach, "peak": derived_upd / 1e9,
                               "unit": "Gupdate/s", "frac": ach / (derived_upd / 1e9), "traffic": None,
                               "probe_peak": upd_s / 1e9, "frac_of_probe": ach / (upd_s / 1e9),
                               "frac_of_single_step_peak": ach / (single_step_upd / 1e9),
                               "peak_src": peak_src}
            else:
                roofs[name] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                               "frac": ach / hbm_peak, "traffic": None, "peak_src": hbm_src}
        return roofs
    roofs = roofs_of(stage_ms, work)
    plain_roofs = roofs_of(plain_stage_ms, dict(ptimer.work))
    # the dominant kernel: the condensation kernel, timed launch by launch
    nl = ptimer.launches["condense"]
    ratio = _traffic_ratio()
    roof = dict(plain_roofs["condense"], kernel="condense_kernel", launches=nl,
                avg_launch_ms=plain_stage_ms["condense"] / max(1, nl),
                traffic=None if ratio is None else ratio * cond_bytes / max(1, nl),
                traffic_unit="bytes per launch",
                algorithmic_bytes_per_launch=cond_bytes / max(1, nl),
                traffic_src=("ncu read + write / algorithmic bytes of the n = 24 capture, scaled to "
                             "the average launch" if ratio is not None else
                             "sources changed since the ncu capture"),
                imad_pipe_active_ncu=CONDENSE_TRAFFIC.get("fmaheavy_active") if ratio is not None else None,
                by_order=by_order,
                frac_of_launch_bound=t_bound / t_meas if t_meas else None,
                timed="CUDA events around each of its launches on the launching stream, plain "
                      "pass over the same batch (the batched form's materialized orders run the "
                      "same kernel)")

    served = None if args.no_served else served_leg(args, mats, value, st)
    kernels = None if args.no_kernels else kernel_leg(st, hbm_peak, mats)
    structured = None if args.no_structured else structured_leg(st, hbm_peak, model_peak(15))

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = OraclePool(mats)
        try:
            el = args.cpu_seconds
            done = len(pool.window(el))
        finally:
            pool.close()
        skipped, workers = pool.skipped, pool.workers
        # every member the oracle finished is also a parity check of the
        # batched form's output for it (identical integers required)
        checked = {i: d == batched_results[i] for i, d in pool.results.items()}
        # the batched GPU form on exactly the members the oracle can reach
        # (like for like with this baseline), CUDA graphs, inputs resident
        small = [pm for pm in mats if oracle_cost(pm) <= 2e6]
        sr = BatchedRunner(small, tune="cache", stream=st)
        sr.upload(st)
        sr.capture(st)
        for _ in range(3):
            sr.compute(st)
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ev.record(st)
        for _ in range(5):
            sr.compute(st)
        b_ev.record(st)
        b_ev.synchronize()
        sr.check_status(st)
        sr.close()
        same_rate = 5 * len(small) / (a_ev.elapsed_time(b_ev) * 1e-3)
        cpu = {"value": done / el, "unit": "exact dets/s", "cores": workers, "kind": "oracle",
               "sample": f"{done} members of the same seeded batch in order, skipping {skipped} whose "
                         f"n^3*prod(n d_v+1) > 2e6, {el:.1f} s, one member per Python process on "
                         f"{workers} cores (small members only: larger ones are out of reach of the oracle)",
               "gpu_output_checked": {"distinct_members": len(checked),
                                      "bit_exact": sum(checked.values()),
                                      "mismatched": [i for i, ok in checked.items() if not ok]},
               "gpu_same_members": {"members": len(small), "exact_dets_per_s": same_rate,
                                    "ratio_to_this_baseline": same_rate / max(done / el, 1e-9),
                                    "note": "the batched form on exactly the cost-capped members the "
                                            "oracle runs (CUDA graphs, inputs resident, L2 not flushed)"}}

    line = {
        "metric": METRIC, "value": value, "unit": "exact dets/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "seed": args.seed, "count": args.count,
                   "form": "batched: per matrix order fused or materialized evaluation + "
                           "condensation (autotuned), CUDA graphs",
                   "mod_p_dets_per_step": modp_per_step, "tuned": tuning,
                   "l2": "flushed before each timed step (256 MiB write, outside the timing)"},
        "mod_p_dets_per_s": modp_value,
        "plain_form": {"value": exact_all / (plain_max * 1e-3), "unit": "exact dets/s",
                       "ms_per_step": plain_max, "identical_output": same,
                       "speedup_of_batched": plain_max / (total_ms / args.steps),
                       "stage_ms": plain_stage_ms, "roofline_by_stage": plain_roofs},
        "roofline": roof,
        "roofline_by_stage": roofs,
        "stage_ms": stage_ms,
        "stage_events": "CUDA events between the per-stage graph launches of every timed step",
        "int_probe": {"imad_per_s": imad_s, "single_step_update_per_s": upd1_s,
                      "pair_element_update_per_s": pair_s, "triple_element_update_per_s": triple_s,
                      "update_per_s_weighted": upd_s},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "exact dets/s", "pipelined": True, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "served": served,
        "hbm_kernels": kernels,
        "structured": structured,
    }
    if rank == 0:
        print(json.dumps(_plain(line)), flush=True)


def _plain(o):
    """JSON-ready copy: numpy scalars and arrays become Python values."""
    import numpy as np
    if isinstance(o, dict):
        return {str(k): _plain(v) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [_plain(v) for v in o]
    if isinstance(o, np.generic):
        return o.item()
    if isinstance(o, np.ndarray):
        return o.tolist()
    return o


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
