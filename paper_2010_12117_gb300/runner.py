"""Prepared determinant jobs: plans, device buffers and pinned host staging
for a fixed list of polynomial matrices, computed by the plain path
(Algorithm 1 per matrix: eval -> condense -> interp per prime chunk, then
CRT), all asynchronous on one stream.

``upload`` copies the inputs from pinned host memory, ``compute`` runs every
stage on the device, ``download`` copies the limbs back; ``results`` turns
them into Python integers.  ``StageTimer`` brackets each library call with
CUDA events on the launching stream so per-kernel time can be attributed.
"""
from __future__ import annotations

from collections import defaultdict
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from .binding import (BATCH_FUSED, BATCH_MATERIALIZE_N, BATCH_MATERIALIZED, EBOUND, Plan,
                      PolydetError, as_u32, limbs_to_ints, tail_entry_words)
from .pipeline import permute_coeffs, prime_count, unpermute_output  # noqa: F401 (re-exported)


class StageTimer:
    """Events around library calls, grouped by stage name, with the
    algorithmic work each call represents."""

    def __init__(self):
        self.events: Dict[str, list] = defaultdict(list)
        self.work: Dict[str, float] = defaultdict(float)
        self.launches: Dict[str, int] = defaultdict(int)
        self.tagged: Dict[tuple, list] = defaultdict(list)  # (name, tag) -> event pairs
        self.tag_work: Dict[tuple, float] = defaultdict(float)

    def run(self, name: str, stream: torch.cuda.Stream, fn, work: float = 0.0, launches: int = 1,
            tag=None):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        self.events[name].append((s, e))
        self.work[name] += work
        self.launches[name] += launches
        if tag is not None:
            self.tagged[(name, tag)].append((s, e))
            self.tag_work[(name, tag)] += work

    def ms(self) -> Dict[str, float]:
        return {k: sum(s.elapsed_time(e) for s, e in v) for k, v in self.events.items()}

    def tag_ms(self, name: str) -> Dict:
        """Per tag of stage ``name``: (milliseconds, work)."""
        return {t: (sum(s.elapsed_time(e) for s, e in v), self.tag_work[(nm, t)])
                for (nm, t), v in self.tagged.items() if nm == name}


def condense_updates(n: int) -> int:
    """Fused modular updates of one n x n elimination: sum_c (n-1-c)^2."""
    return (n - 1) * n * (2 * n - 1) // 6


class PlainRunner:
    def __init__(self, mats: Sequence, nprimes: Optional[Sequence[int]] = None,
                 budget_bytes: int = 6 << 30, device: str = "cuda", full_grid: bool = False):
        self.mats = list(mats)
        self.plans: List[Plan] = []
        for i, pm in enumerate(self.mats):
            P = nprimes[i] if nprimes is not None else prime_count(pm.coeffs)
            self.plans.append(Plan(pm.n, pm.degs, P, full_grid=full_grid))
        self.dev = torch.device(device)
        co, ro, lo = [0], [0], [0]
        for pm, pl in zip(self.mats, self.plans):
            co.append(co[-1] + pm.n * pm.n * pl.E)
            ro.append(ro[-1] + pl.P * pl.C)
            lo.append(lo[-1] + pl.C * pl.W)
        self.coef_off, self.res_off, self.limb_off = co, ro, lo
        # prime chunks per job under the scratch budget
        self.chunks: List[List[tuple]] = []
        max_ev = max_dv = max_ws = 1
        for pm, pl in zip(self.mats, self.plans):
            per = 4 * (pm.n * pm.n * pl.G + pl.G + max(pl.eval_ws_words, pl.interp_ws_words))
            ch = max(1, min(pl.P, budget_bytes // per))
            self.chunks.append([(a, min(pl.P, a + ch)) for a in range(0, pl.P, ch)])
            max_ev = max(max_ev, ch * pm.n * pm.n * pl.G)
            max_dv = max(max_dv, ch * pl.G)
            max_ws = max(max_ws, ch * max(pl.eval_ws_words, pl.interp_ws_words))
        self.coeffs_dev = torch.empty(co[-1], dtype=torch.int32, device=self.dev)
        self.residues = torch.empty(max(ro[-1], 1), dtype=torch.int32, device=self.dev)
        self.limbs = torch.empty(max(lo[-1], 1), dtype=torch.int32, device=self.dev)
        self.evals = torch.empty(max_ev, dtype=torch.int32, device=self.dev)
        self.detvals = torch.empty(max_dv, dtype=torch.int32, device=self.dev)
        self.ws = torch.empty(max_ws, dtype=torch.int32, device=self.dev)
        self.host_in = torch.empty(co[-1], dtype=torch.int32, pin_memory=True)
        self.host_out = torch.empty(max(lo[-1], 1), dtype=torch.int32, pin_memory=True)
        for i, pm in enumerate(self.mats):
            self.host_in[co[i]:co[i + 1]] = torch.from_numpy(
                np.ascontiguousarray(pm.coeffs, dtype=np.int32).reshape(-1))

    # -- sizes ---------------------------------------------------------------
    @property
    def h2d_bytes(self) -> int:
        return 4 * self.coef_off[-1]

    @property
    def d2h_bytes(self) -> int:
        return 4 * self.limb_off[-1]

    def modp_dets(self) -> int:
        return sum(pl.P * pl.G for pl in self.plans)

    def kernel_launches(self) -> int:
        tot = 0
        for pl, chunks in zip(self.plans, self.chunks):
            tot += len(chunks) * (2 * pl.k + 1) + 1
        return tot

    # -- the three phases ----------------------------------------------------
    def upload(self, stream: torch.cuda.Stream) -> None:
        with torch.cuda.stream(stream):
            self.coeffs_dev.copy_(self.host_in, non_blocking=True)

    def compute(self, stream: torch.cuda.Stream, timer: Optional[StageTimer] = None) -> None:
        for i, (pm, pl) in enumerate(zip(self.mats, self.plans)):
            c = self.coeffs_dev[self.coef_off[i]:self.coef_off[i + 1]]
            res = self.residues[self.res_off[i]:self.res_off[i + 1]]
            n2 = pm.n * pm.n
            for lo, hi in self.chunks[i]:
                np_ = hi - lo
                r = res[lo * pl.C:hi * pl.C]
                calls = [
                    ("eval", lambda: pl.eval(c, lo, hi, self.evals, self.ws, stream),
                     4.0 * np_ * n2 * (pl.E + pl.G), pl.k),
                    ("condense", lambda: pl.condense(self.evals, lo, hi, self.detvals, stream),
                     float(np_ * pl.G * condense_updates(pm.n)), 1),
                    ("interp", lambda: pl.interp(self.detvals, lo, hi, r, self.ws, stream),
                     4.0 * np_ * (pl.G + pl.C), pl.k),
                ]
                for name, fn, work, nl in calls:
                    if timer is None:
                        fn()
                    else:
                        timer.run(name, stream, fn, work, nl, tag=pm.n)
            lb = self.limbs[self.limb_off[i]:self.limb_off[i + 1]]
            fn = lambda: pl.crt(res, lb, stream)  # noqa: E731
            if timer is None:
                fn()
            else:
                timer.run("crt", stream, fn, 4.0 * pl.C * (pl.P + pl.W), 1)

    def download(self, stream: torch.cuda.Stream) -> None:
        with torch.cuda.stream(stream):
            self.host_out.copy_(self.limbs, non_blocking=True)

    def check_status(self, stream: torch.cuda.Stream) -> None:
        for pl in self.plans:
            st = pl.sync_status(stream)
            if st:
                raise PolydetError(EBOUND, f"device status {st:#x}")

    def results(self) -> List[List[int]]:
        out = []
        host = self.host_out.numpy().view(np.uint32)
        for i, pl in enumerate(self.plans):
            out.append(limbs_to_ints(host[self.limb_off[i]:self.limb_off[i + 1]].reshape(pl.C, pl.W), pl.W))
        return out

    def close(self) -> None:
        for pl in self.plans:
            pl.close()


def variable_order(n: int, degs: Sequence[int]) -> List[int]:
    """The order the batched form runs a job's variables in: the one of
    lowest degree first when its matrix order is materialized by default (the
    first variable's pass writes every evaluated matrix, and a short input is
    the cheapest to transform), last when fused (the last variable is the
    one evaluated inside the determinant kernel).  Ties keep the given order
    in the first case and come out reversed in the second."""
    order = sorted(range(len(degs)), key=lambda v: (int(degs[v]), v))
    return order if n >= BATCH_MATERIALIZE_N else order[::-1]


class BatchedRunner:
    """The batched form: every job of the list in one run of four stages
    (partial evaluation; per matrix order either one persistent fused
    evaluation + condensation kernel or materialized chunks of evaluated
    matrices and the condensation kernel; interpolation; CRT), optionally
    captured once in CUDA graphs and replayed."""

    def __init__(self, mats: Sequence, nprimes: Optional[Sequence[int]] = None,
                 device: str = "cuda", tune=True, stream: Optional[torch.cuda.Stream] = None,
                 full_grid: bool = False):
        from .binding import Batch
        self.mats = list(mats)
        Ps = [nprimes[i] if nprimes is not None else prime_count(pm.coeffs)
              for i, pm in enumerate(self.mats)]
        # every job runs with its variables in variable_order(); results()
        # puts the output coefficients back in the caller's order
        self.orders = [variable_order(pm.n, pm.degs) for pm in self.mats]
        self.batch = Batch([(pm.n, tuple(pm.degs[v] for v in o), P)
                            for pm, o, P in zip(self.mats, self.orders, Ps)], full_grid=full_grid)
        self.dev = torch.device(device)
        w = self.batch.words
        self.coeffs_dev = torch.empty(max(1, w["coeffs"]), dtype=torch.int32, device=self.dev)
        self.partial = torch.empty(max(1, w["partial"]), dtype=torch.int32, device=self.dev)
        self.detvals = torch.empty(max(1, w["detvals"]), dtype=torch.int32, device=self.dev)
        self.residues = torch.empty(max(1, w["residues"]), dtype=torch.int32, device=self.dev)
        self.limbs = torch.empty(max(1, w["limbs"]), dtype=torch.int32, device=self.dev)
        self.ws = torch.empty(max(1, w["workspace"]), dtype=torch.int32, device=self.dev)
        self.host_in = torch.empty(max(1, w["coeffs"]), dtype=torch.int32, pin_memory=True)
        self.host_out = torch.empty(max(1, w["limbs"]), dtype=torch.int32, pin_memory=True)
        co = self.batch.offsets["coeffs"]
        for i, pm in enumerate(self.mats):
            c = permute_coeffs(pm.coeffs, pm.degs, self.orders[i])
            self.host_in[co[i]:co[i + 1]] = torch.from_numpy(np.ascontiguousarray(c, dtype=np.int32).reshape(-1))
        self.graph = None
        self.tuning = {}
        st = stream or torch.cuda.current_stream()
        if tune == "cache":  # apply earlier choices of the autotuner, search nothing
            from .tune import apply_cached
            self.tuning = apply_cached(self.batch)
        elif tune:
            self.upload(st)
            from .tune import tune as _tune
            self.tuning = _tune(self.batch, self.coeffs_dev, self.partial, self.detvals,
                                self._workspace, st)
        self._workspace(self.batch.words["workspace"])

    def set_chunk_words(self, words: int) -> None:
        """Budget of one materialized chunk (words of evaluated matrices)."""
        self.batch.set_chunk_words(words)
        self.graph = None
        self._workspace(self.batch.words["workspace"])

    def set_modes(self, modes) -> None:
        """Mode of every order (an int) or of some ({n: mode}); stage 1 must
        run again afterwards (compute() does)."""
        orders = self.batch.orders()
        items = modes.items() if isinstance(modes, dict) else ((n, modes) for n in orders)
        for n, m in items:
            self.batch.set_mode(n, m)
        self.graph = None
        self._workspace(self.batch.words["workspace"])

    def _workspace(self, words: int) -> torch.Tensor:
        """The workspace, grown to at least ``words`` (modes change its size)."""
        if self.ws.numel() < words:
            self.ws = torch.empty(words, dtype=torch.int32, device=self.dev)
        return self.ws

    @property
    def h2d_bytes(self) -> int:
        return 4 * self.batch.words["coeffs"]

    @property
    def d2h_bytes(self) -> int:
        return 4 * self.batch.words["limbs"]

    def modp_dets(self) -> int:
        return sum(int(i.P) * int(i.G) for i in self.batch.job_info)

    def updates(self) -> int:
        return sum(int(i.P) * int(i.G) * condense_updates(int(i.n)) for i in self.batch.job_info)

    def kernel_launches(self) -> int:
        tot = 0
        for i in self.batch.job_info:
            n, k, P, G = int(i.n), int(i.nvars), int(i.P), int(i.G)
            tot += max(1, k - 1)             # stage 1 passes (or the repack / reduction)
            if self.batch.mode(n) == BATCH_MATERIALIZED:
                Gs = tail_entry_words(tuple(i.M[:k]))
                cp = max(1, min(P, int(self.batch.info.chunk_words) // (n * n * Gs)))
                tot += 2 * (-(-P // cp))     # first-variable pass + condensation per chunk
            tot += k + 1                     # interpolation passes and CRT
        fused = [n for n in self.batch.orders() if self.batch.mode(n) == BATCH_FUSED]
        return tot + len(fused)

    def upload(self, stream: torch.cuda.Stream) -> None:
        with torch.cuda.stream(stream):
            self.coeffs_dev.copy_(self.host_in, non_blocking=True)

    def _stages(self, stream):
        b = self.batch
        return [("eval", lambda: b.eval(self.coeffs_dev, self.partial, self.ws, stream),
                 4.0 * (b.words["coeffs"] + b.words["partial"])),
                ("condense", lambda: b.condense(self.partial, self.detvals, self.ws, stream),
                 float(self.updates())),
                ("interp", lambda: b.interp(self.detvals, self.residues, self.ws, stream),
                 4.0 * (b.words["detvals"] + b.words["residues"])),
                ("crt", lambda: b.crt(self.residues, self.limbs, stream),
                 4.0 * (b.words["residues"] + b.words["limbs"]))]

    def capture(self, stream: torch.cuda.Stream) -> None:
        """Capture each stage of one run in its own CUDA graph; compute()
        then replays the four graphs (stage events go between them)."""
        for _, fn, _ in self._stages(stream):  # warm: kernel attributes set before capture
            fn()
        stream.synchronize()
        graphs = []
        for name, _, work in self._stages(stream):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                cur = torch.cuda.current_stream()
                dict((n, f) for n, f, _ in self._stages(cur))[name]()
            graphs.append((name, g, work))
        self.graph = graphs

    def compute(self, stream: torch.cuda.Stream, timer: Optional[StageTimer] = None) -> None:
        if self.graph is not None:
            with torch.cuda.stream(stream):
                for name, g, work in self.graph:
                    if timer is None:
                        g.replay()
                    else:
                        timer.run(name, stream, g.replay, work)
            return
        for name, fn, work in self._stages(stream):
            if timer is None:
                fn()
            else:
                timer.run(name, stream, fn, work)

    def download(self, stream: torch.cuda.Stream) -> None:
        self._last_host = self.host_out
        with torch.cuda.stream(stream):
            self.host_out.copy_(self.limbs, non_blocking=True)

    def run_pipelined(self, steps: int, stream: torch.cuda.Stream,
                      copy_stream: Optional[torch.cuda.Stream] = None) -> None:
        """``steps`` full runs end to end - upload of the inputs from pinned
        host memory, compute, download of the limbs to pinned host memory -
        with each run's download overlapping the next run's compute: the
        limbs go to one of two device staging buffers (a device copy) and
        from there to host on ``copy_stream``.  Returns after everything has
        landed; results() then reads the last run's limbs."""
        cs = copy_stream or torch.cuda.Stream()
        if getattr(self, "_stage", None) is None:
            self._stage = [torch.empty_like(self.limbs) for _ in range(2)]
            self._host2 = [self.host_out, torch.empty_like(self.host_out, pin_memory=True)]
        free = [None, None]  # copy-stream events: staging slot read out
        for k in range(steps):
            slot = k % 2
            self.upload(stream)
            self.compute(stream)
            if free[slot] is not None:
                stream.wait_event(free[slot])
            with torch.cuda.stream(stream):
                self._stage[slot].copy_(self.limbs, non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(stream)
            cs.wait_event(ready)
            with torch.cuda.stream(cs):
                self._host2[slot].copy_(self._stage[slot], non_blocking=True)
            free[slot] = torch.cuda.Event()
            free[slot].record(cs)
        cs.synchronize()
        stream.synchronize()
        if steps:
            self._last_host = self._host2[(steps - 1) % 2]

    def check_status(self, stream: torch.cuda.Stream) -> None:
        st = self.batch.sync_status(stream)
        if st:
            raise PolydetError(EBOUND, f"device status {st:#x}")

    def results(self) -> List[List[int]]:
        out = []
        host = getattr(self, "_last_host", self.host_out).numpy().view(np.uint32)
        lo = self.batch.offsets["limbs"]
        for j, info in enumerate(self.batch.job_info):
            C, W = int(info.C), int(info.W)
            vals = limbs_to_ints(host[lo[j]:lo[j + 1]].reshape(C, W), W)
            order = self.orders[j]
            box = tuple(int(info.D[v]) + 1 for v in range(len(order)))
            out.append(unpermute_output(vals, order, box))  # the caller's variable order
        return out

    def release_buffers(self) -> None:
        """Return the device buffers to torch's caching allocator (stream
        ordered, no device synchronisation); the batch's small plan tables
        stay until close()."""
        self.graph = None
        for name in ("coeffs_dev", "partial", "detvals", "residues", "limbs", "ws", "_stage"):
            setattr(self, name, None)

    def close(self) -> None:
        self.release_buffers()
        self.batch.close()
