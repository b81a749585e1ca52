"""Run-time and device-memory prediction for determinant jobs.

The paper predicts the run time of a job as T = C_p r^2 Round(mean T_e, 2) mu
(Sec. 5): primes x entries x the mean per-entry FFT time x a replication
factor.  Here the same idea is carried to the batched GPU form in two layers:

* ``analytic`` - a bound from the job's shape alone: prime count from the
  Hadamard bound, grid and output sizes, the exact buffer bytes of the
  batched form (memory), and a roofline time, max(updates / integer-pipe
  rate, bytes / HBM rate) plus a per-launch cost, each the smaller over the
  two modes of the batched form.  It needs no training and is a lower bound
  of both quantities.
* ``Predictor`` - an fp32 MLP 8 -> 64 -> 64 -> 2 trained on the method's own
  measured timings and footprints, with forward, backward and Adam in the
  library's CUDA kernels.  Inputs: n, k, max and mean degree, density,
  coefficient bits, and the logs of the analytic time and memory; outputs:
  log(measured / analytic) for time and memory (standardised), a correction
  to the bound, so that a network with a constant output reproduces the
  calibrated bound and training adds what the shape tells beyond it.  The
  analytic bound judges it:
  a prediction below the bound is raised to it, one more than ``max_ratio``
  times the larger of the bound and the smallest measured value falls back
  to the bound times the calibrated median ratio, and an untrained predictor
  answers with that calibrated bound.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding

UPDATE_RATE = 3.0e12      # fused updates/s, the probe's ceiling on GB300
HBM_RATE = 6.786e12       # bytes/s, measured copy bandwidth
LAUNCH_S = 4e-6           # per kernel launch inside a graph


def _nextpow2(x: int) -> int:
    n = 1
    while n < x:
        n *= 2
    return n


@dataclass
class Shape:
    n: int
    degs: tuple
    P: int
    density: float
    coef_bits: float

    @property
    def k(self) -> int:
        return len(self.degs)


def shape_of(pm) -> Shape:
    from .pipeline import prime_count
    c = np.asarray(pm.coeffs)
    nz = float((c != 0).mean()) if c.size else 0.0
    bits = math.log2(float(np.abs(c).max(initial=0)) + 1.0)
    return Shape(pm.n, tuple(int(d) for d in pm.degs), prime_count(c), nz, bits)


_LIMBS = {}


def _limbs(P: int) -> int:
    """32-bit words of the product of the first P primes (the CRT output width)."""
    if P not in _LIMBS:
        _LIMBS[P] = (math.prod(binding.prime_table()[:P]).bit_length() + 31) // 32
    return _LIMBS[P]


def default_mode(n: int) -> int:
    """The batched form's mode of order n when nothing was tuned."""
    return binding.BATCH_MATERIALIZED if n >= binding.BATCH_MATERIALIZE_N else binding.BATCH_FUSED


def analytic_mode(s: Shape, mode: int) -> tuple:
    """(seconds, bytes) of one job alone in the batched form in ``mode``:
    the exact buffer bytes the library lays out (coefficients, partial
    tensor sized for either mode, determinant values, residues, limbs,
    workspace) and a roofline time, max(updates / integer-pipe rate,
    bytes / HBM rate) plus a per-launch cost."""
    from .runner import variable_order
    n, k, P = s.n, s.k, s.P
    degs = tuple(s.degs[v] for v in variable_order(n, s.degs))  # the batched form's order
    D = [n * d for d in degs]
    M = [x + 1 for x in D]  # evaluation nodes per variable (node grid)
    G = math.prod(M)
    C = math.prod(x + 1 for x in D)
    E = math.prod(d + 1 for d in degs)
    L = degs[-1] + 1
    Lp = _nextpow2(L)
    rows = G // M[-1]
    W = _limbs(P)
    n2 = n * n

    def words_after(v):  # per entry, after the passes of the variables > v
        return math.prod((degs[u] + 1) if u <= v else M[u] for u in range(k))
    fused_part = P * rows * n2 * Lp
    mat_part = P * n2 * words_after(0)
    partial = -(-max(fused_part, mat_part) // 8) * 8
    iws = 0
    for v in range(1, k):
        sz = 1
        for u in range(k):
            sz *= M[u] if u < v else (D[u] + 1)
        iws = max(iws, sz)
    scratch = P * 2 * iws
    chunk = 0
    if mode == binding.BATCH_FUSED:
        pws = 0
        if k > 2:
            for v in range(1, k - 1):
                sz = L
                for u in range(k - 1):
                    sz *= (degs[u] + 1) if u < v else M[u]
                pws = max(pws, sz)
            pws *= 2 * n2
        scratch = max(scratch, P * pws)
        moved = 4 * (2 * fused_part + 2 * P * G + P * C + C * W)
        launches = max(1, k - 1) + k + 2
    else:
        hws = max([words_after(v - 1) for v in range(2, k, 2)], default=0) * n2 * P
        Gs = binding.tail_entry_words(M)
        cp = max(1, min(P, binding.BATCH_CHUNK_WORDS // (n2 * Gs)))
        scratch = max(scratch, hws)
        chunk = -(-(cp * n2 * Gs) // 64) * 64
        moved = 4 * (2 * mat_part + 2 * P * n2 * G + 2 * P * G + P * C + C * W)
        launches = max(1, k - 1) + 2 * (-(-P // cp)) + k + 1
    # the workspace: 4 fan-out scratch slices or two chunk buffers, whichever is larger
    ws = max(4 * (-(-scratch // 64) * 64), 2 * chunk)
    words = n2 * E + partial + P * G + P * C + C * W + 256 + ws
    updates = P * G * (n - 1) * n * (2 * n - 1) // 6
    t = max(updates / UPDATE_RATE, moved / HBM_RATE) + launches * LAUNCH_S
    return t, float(4 * words)


def analytic(s: Shape) -> tuple:
    """(seconds, bytes): a lower bound of both in whichever mode runs."""
    a = analytic_mode(s, binding.BATCH_FUSED)
    b = analytic_mode(s, binding.BATCH_MATERIALIZED)
    return min(a[0], b[0]), min(a[1], b[1])


def features(s: Shape) -> np.ndarray:
    t, m = analytic_mode(s, default_mode(s.n))
    return np.array([s.n / 32.0, s.k / 6.0, max(s.degs) / 8.0, float(np.mean(s.degs)) / 8.0,
                     s.density, s.coef_bits / 32.0, math.log10(t) / 4.0 + 1.0, math.log2(m) / 40.0],
                    dtype=np.float32)


class Predictor:
    """The MLP, its training loop and the analytic judge."""

    def __init__(self, seed: int = 0, device: str = "cuda", max_ratio: float = 50.0):
        self.dev = torch.device(device)
        self.params = torch.from_numpy(init_params(seed)).to(self.dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.mu = np.zeros(2, dtype=np.float32)
        self.sd = np.ones(2, dtype=np.float32)
        self.ratio = np.ones(2, dtype=np.float64)  # calibrated median actual / bound
        self.floor = np.zeros(2, dtype=np.float64)  # smallest measured (seconds, bytes)
        self.trained = False
        self.max_ratio = max_ratio

    # -- training ----------------------------------------------------------
    def fit(self, X: np.ndarray, Y: np.ndarray, bounds: np.ndarray, steps: int = 1500,
            lr: float = 3e-3, weight_decay: float = 1e-4) -> List[float]:
        """X [B][8] features, Y [B][2] measured (seconds, bytes), bounds [B][2]
        analytic (seconds, bytes).  Full-batch Adam on the GPU kernels."""
        logy = np.log(np.maximum(Y, 1e-12)).astype(np.float64)
        logr = logy - np.log(np.maximum(bounds, 1e-12))  # the correction to the bound
        self.mu = logr.mean(0).astype(np.float32)
        self.sd = np.maximum(logr.std(0), 1e-3).astype(np.float32)
        self.ratio = np.exp(np.median(logr, axis=0))
        self.floor = np.min(Y, axis=0).astype(np.float64)
        T = ((logr - self.mu) / self.sd).astype(np.float32)
        B = len(X)
        x = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(self.dev)
        t = torch.from_numpy(np.ascontiguousarray(T)).to(self.dev)
        y = torch.empty(B, 2, device=self.dev)
        act = torch.empty(B, 128, device=self.dev)
        delta = torch.empty(B, 130, device=self.dev)
        grads = torch.empty(binding.MLP_PARAMS, device=self.dev)
        loss = torch.empty(1, device=self.dev)
        hist = []
        for it in range(steps):
            binding.mlp_forward(self.params, x, y, act)
            binding.mlp_backward(self.params, x, t, y, act, delta, grads, loss)
            self.step += 1
            binding.mlp_adam(self.params, grads, self.m, self.v, self.step, lr,
                             weight_decay=weight_decay)
            if it % 100 == 0 or it == steps - 1:
                hist.append(float(loss.item()))
        self.trained = True
        return hist

    # -- inference -----------------------------------------------------------
    def raw(self, X: np.ndarray, bounds: np.ndarray) -> np.ndarray:
        """MLP outputs mapped back to (seconds, bytes) for jobs with analytic
        bounds ``bounds`` [len][2], unjudged."""
        x = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(self.dev)
        y = torch.empty(len(X), 2, device=self.dev)
        binding.mlp_forward(self.params, x, y, None)
        out = y.cpu().numpy().astype(np.float64) * self.sd + self.mu
        return np.asarray(bounds, dtype=np.float64) * np.exp(out)

    def predict(self, shapes: Sequence[Shape]) -> np.ndarray:
        """Judged predictions [len][2] = (seconds, bytes)."""
        bounds = np.array([analytic(s) for s in shapes], dtype=np.float64)
        if not self.trained or len(shapes) == 0:
            return bounds * self.ratio
        X = np.stack([features(s) for s in shapes])
        pred = self.raw(X, bounds)
        pred = np.maximum(pred, bounds)
        # implausibly large: more than max_ratio times the bound, or than the
        # smallest footprint / time ever measured when the bound is below it
        # (allocator granularity and launch latency put a floor under both)
        bad = pred > self.max_ratio * np.maximum(bounds, self.floor)
        pred[bad] = (bounds * self.ratio)[bad]
        return pred


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases, in the flat layout of polydet.h."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((8, 64), (64, 64), (64, 2)):
        lim = math.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, (fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)
