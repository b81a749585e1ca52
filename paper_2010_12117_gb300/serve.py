"""Continuous batching of polynomial-determinant requests on one GPU.

Requests arrive over time (seeded Poisson stream).  The loop keeps up to
``slots`` waves in flight, each on its own CUDA stream: whenever a slot is
free it forms a wave from the requests that have arrived - shortest predicted
run time first, requests that have waited longest jumped ahead - admitting
while the predicted device memory of everything in flight stays within the
budget and the wave's predicted time stays within ``wave_seconds`` (up to
``backlog_factor`` times that while the queue holds more predicted work than
the slots can start at the target).  A wave
is one batched run (fused kernels, no host synchronisation inside); its limbs
come back asynchronously and the loop notices completion through an event.
Freed buffers go back to torch's stream-ordered caching allocator, so a
finishing wave does not synchronise the device while others run; the plan
tables of finished waves are destroyed once the device is idle.

A request's result does not depend on which wave it ran in: every job keeps
its own plan (primes, grid) and buffers inside a wave.  When a wave
completes, its device status word is read before anything is returned; a
wave whose word is set returns no results, and its jobs are counted as
failed.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from .predictor import Predictor, Shape, analytic, features, shape_of
from .runner import BatchedRunner


@dataclass
class Done:
    idx: int
    arrival: float
    start: float
    finish: float
    coeffs: List[int]
    wave: int
    ok: bool = True  # False: the wave's device status word was set; no result


@dataclass
class ServeReport:
    jobs: int
    waves: int
    wall_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    exact_dets_per_s: float
    modp_dets: int
    peak_pred_mem: float
    done: List[Done] = field(default_factory=list)
    failed: int = 0  # jobs of waves whose device status word was set
    host_launch_s: float = 0.0  # host time spent planning and enqueueing waves

    def summary(self) -> dict:
        return {"jobs": int(self.jobs), "waves": int(self.waves), "wall_s": float(self.wall_s),
                "p50_ms": float(self.p50_ms), "p99_ms": float(self.p99_ms), "mean_ms": float(self.mean_ms),
                "exact_dets_per_s": float(self.exact_dets_per_s), "modp_dets": int(self.modp_dets),
                "peak_predicted_mem_bytes": float(self.peak_pred_mem), "failed_jobs": int(self.failed),
                "host_launch_s": float(self.host_launch_s)}


def measure(pm, stream: torch.cuda.Stream, reps: int = 2) -> tuple:
    """Run one job alone in the batched form: (seconds, device bytes)."""
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    r = BatchedRunner([pm], tune="cache", stream=stream)
    free1 = torch.cuda.mem_get_info()[0]
    r.upload(stream)
    r.compute(stream)
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(reps):
        r.compute(stream)
    e.record(stream)
    e.synchronize()
    sec = s.elapsed_time(e) / reps * 1e-3
    r.close()
    return sec, float(max(free0 - free1, 1))


def calibrate(mats: Sequence, stream: Optional[torch.cuda.Stream] = None, reps: int = 2):
    """Timings and footprints the method itself generates, for training:
    returns (features [B][8], measured [B][2], bounds [B][2]); each time is
    the mean of ``reps`` runs after a warm one."""
    st = stream or torch.cuda.Stream()
    measure(mats[0], st)  # warm-up: module load, kernel attributes
    X, Y, Bd = [], [], []
    for pm in mats:
        s = shape_of(pm)
        X.append(features(s))
        Y.append(measure(pm, st, reps=reps))
        Bd.append(analytic(s))
    return np.stack(X), np.array(Y, dtype=np.float64), np.array(Bd, dtype=np.float64)


class Server:
    def __init__(self, predictor: Optional[Predictor], mem_budget: float, slots: int = 2,
                 wave_seconds: float = 0.05, max_wave_jobs: int = 128, max_wait: float = 0.25,
                 backlog_factor: float = 4.0):
        self.pred = predictor or Predictor()
        self.mem_budget = float(mem_budget)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.wave_seconds = wave_seconds
        self.max_wave_jobs = max_wave_jobs
        self.max_wait = max_wait
        self.backlog_factor = backlog_factor

    def run(self, arrivals: Sequence, keep_results: bool = True) -> ServeReport:
        shapes: List[Shape] = [shape_of(a.job) for a in arrivals]
        preds = self.pred.predict(shapes)  # [len][2]: seconds, bytes
        order = sorted(range(len(arrivals)), key=lambda i: arrivals[i].t)
        pending: deque = deque()
        nxt = 0
        inflight: List[dict] = []
        free_slots = list(range(len(self.streams)))
        graveyard: List[BatchedRunner] = []
        done: List[Done] = []
        mem_used = 0.0
        peak = 0.0
        waves = 0
        modp = 0
        failed = 0
        host_launch = 0.0
        t0 = time.perf_counter()
        while nxt < len(order) or pending or inflight:
            now = time.perf_counter() - t0
            while nxt < len(order) and arrivals[order[nxt]].t <= now:
                pending.append(order[nxt])
                nxt += 1
            # completions
            for w in list(inflight):
                if w["event"].query():
                    fin = time.perf_counter() - t0
                    # the wave's stream is idle: reading its status word is
                    # one small copy; a set word (a bounded wait that ran
                    # out, a degree bound that did not hold) means its limbs
                    # are not the determinants, so none is returned
                    status = w["runner"].batch.sync_status(self.streams[w["slot"]])
                    if status:
                        failed += len(w["jobs"])
                        res = [[] for _ in w["jobs"]]
                    else:
                        res = w["runner"].results() if keep_results else [[] for _ in w["jobs"]]
                    for j, coeffs in zip(w["jobs"], res):
                        done.append(Done(j, arrivals[j].t, w["start"], fin, coeffs, w["id"],
                                         ok=not status))
                    w["runner"].release_buffers()
                    graveyard.append(w["runner"])
                    mem_used -= w["mem"]
                    free_slots.append(w["slot"])
                    inflight.remove(w)
            if not inflight and graveyard:
                for r in graveyard:
                    r.close()
                graveyard.clear()
            # admission
            if free_slots and pending:
                now = time.perf_counter() - t0
                waiting = sorted(pending, key=lambda j: (0 if now - arrivals[j].t > self.max_wait else 1,
                                                         preds[j][0]))
                # a backlog larger than the slots can start at the wave target
                # gets waves up to backlog_factor times longer (fewer, larger
                # batched runs: more jobs per launch), sized so that the slots
                # share it
                backlog = float(sum(preds[j][0] for j in pending))
                limit = self.wave_seconds
                if backlog > self.wave_seconds * len(self.streams):
                    limit = min(self.backlog_factor * self.wave_seconds, backlog / len(self.streams))
                wave, wt, wm = [], 0.0, 0.0
                for j in waiting:
                    if len(wave) >= self.max_wave_jobs:
                        break
                    t_j, m_j = preds[j]
                    fits_mem = mem_used + wm + m_j <= self.mem_budget
                    alone = not wave and not inflight  # too big for the budget: run it by itself
                    if (fits_mem or alone) and (not wave or wt + t_j <= limit):
                        wave.append(j)
                        wt += t_j
                        wm += m_j
                if wave:
                    for j in wave:
                        pending.remove(j)
                    slot = free_slots.pop()
                    st = self.streams[slot]
                    start = time.perf_counter() - t0
                    runner = BatchedRunner([arrivals[j].job for j in wave], nprimes=[shapes[j].P for j in wave],
                                           tune="cache", stream=st)
                    runner.upload(st)
                    runner.compute(st)
                    runner.download(st)
                    ev = torch.cuda.Event()
                    ev.record(st)
                    host_launch += time.perf_counter() - t0 - start
                    modp += runner.modp_dets()
                    inflight.append({"id": waves, "jobs": wave, "runner": runner, "event": ev,
                                     "mem": wm, "slot": slot, "start": start})
                    waves += 1
                    mem_used += wm
                    peak = max(peak, mem_used)
                    continue
            # nothing to do right now: wait for the next arrival or completion
            if inflight:
                time.sleep(5e-5)
            elif nxt < len(order):
                time.sleep(max(0.0, min(1e-3, arrivals[order[nxt]].t - (time.perf_counter() - t0))))
        for r in graveyard:
            r.close()
        wall = max((d.finish for d in done), default=0.0) - min((arrivals[i].t for i in order), default=0.0)
        lat = np.array([1e3 * (d.finish - d.arrival) for d in done])
        done.sort(key=lambda d: d.idx)
        return ServeReport(len(done), waves, wall, float(np.percentile(lat, 50)),
                           float(np.percentile(lat, 99)), float(lat.mean()),
                           len(done) / max(wall, 1e-9), modp, peak, done, failed, host_launch)
