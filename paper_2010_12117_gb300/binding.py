"""Thin ctypes binding of libpolydet (``include/polydet.h``).

Argument marshalling only: every stage of the determinant runs in the
library's CUDA kernels.  Device buffers are torch CUDA tensors (int32
storage; residues are reinterpreted as uint32), streams are torch streams.
If the library has not been built this module raises on first use; there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libpolydet.so")

MAX_VARS = 6
OK, EINVAL, EDEGREE, EPRIMES, ENOMEM, ECUDA, ETIMEOUT, EBOUND = 0, -1, -2, -3, -4, -5, -6, -7
ETOOBIG = -8
STATIC_SCRATCH_WORDS = 4 * 1024 * 1024
_ERRNAMES = {EINVAL: "EINVAL", EDEGREE: "EDEGREE", EPRIMES: "EPRIMES", ENOMEM: "ENOMEM",
             ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT", EBOUND: "EBOUND", ETOOBIG: "ETOOBIG"}


class PolydetError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what} failed: {_ERRNAMES.get(code, code)} {last_error()}")


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nvars", ctypes.c_int32), ("P", ctypes.c_int32),
                ("W", ctypes.c_int32), ("E", ctypes.c_int64), ("G", ctypes.c_int64),
                ("C", ctypes.c_int64), ("d", ctypes.c_int32 * MAX_VARS),
                ("D", ctypes.c_int32 * MAX_VARS), ("N", ctypes.c_int32 * MAX_VARS),
                ("eval_ws_words", ctypes.c_uint64), ("interp_ws_words", ctypes.c_uint64),
                ("M", ctypes.c_int32 * MAX_VARS), ("flags", ctypes.c_uint32),
                ("entries", ctypes.c_int32), ("unique", ctypes.c_int32)]


MAX_N = 32
OFF_COEFFS, OFF_PARTIAL, OFF_DETVALS, OFF_RESIDUES, OFF_LIMBS = 0, 1, 2, 3, 4


FLAG_FULL_GRID = 0x1
BATCH_FUSED = 0
BATCH_MATERIALIZED = 1
BATCH_MATERIALIZE_N = 14
BATCH_CHUNK_WORDS = 512 * 1024 * 1024


class Job(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nvars", ctypes.c_int32), ("nprimes", ctypes.c_int32),
                ("d", ctypes.c_int32 * MAX_VARS), ("flags", ctypes.c_uint32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("njobs", ctypes.c_int32), ("coeff_words", ctypes.c_int64),
                ("partial_words", ctypes.c_int64), ("detval_words", ctypes.c_int64),
                ("residue_words", ctypes.c_int64), ("limb_words", ctypes.c_int64),
                ("workspace_words", ctypes.c_uint64), ("items", ctypes.c_int64 * (MAX_N + 1)),
                ("threads", ctypes.c_int32 * (MAX_N + 1)), ("blocks", ctypes.c_int32 * (MAX_N + 1)),
                ("mode", ctypes.c_int32 * (MAX_N + 1)), ("chunk_words", ctypes.c_uint64)]


_lib = None

# name -> (restype, argtypes); the exported C ABI.
_VP, _I, _U32, _PI32, _PU32, _PI64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32,
                                      ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_uint32),
                                      ctypes.POINTER(ctypes.c_int64))
SIGNATURES = {
    "polydet_prime_table": (_I, [_PU32]),
    "polydet_hadamard_primes": (_I, [_I, _PI64, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_double)]),
    "polydet_plan": (_I, [ctypes.POINTER(_VP), _I, _I, _PI32, _I, _U32]),
    "polydet_plan_degrees": (_I, [ctypes.POINTER(_VP), _I, _I, _PI32, _PI32, _I, _U32]),
    "polydet_det_degree_bound": (_I, [_I, _I, _PI32, _PI32]),
    "polydet_unique_entries": (_I, [_I, ctypes.c_int64, _PI32, _PI32, _PI32, _PI32]),
    "polydet_plan_set_entry_map": (_I, [_VP, _PI32, _I]),
    "polydet_stream_ws_words": (ctypes.c_uint64, [_VP, _I]),
    "polydet_eval_condense": (_I, [_VP, _VP, _I, _I, _VP, _VP, ctypes.c_uint64, _VP]),
    "polydet_plan_destroy": (_I, [_VP]),
    "polydet_plan_cache_clear": (_I, []),
    "polydet_plan_query": (_I, [_VP, ctypes.POINTER(PlanInfo)]),
    "polydet_plan_primes": (_I, [_VP, _PU32]),
    "polydet_plan_roots": (_I, [_VP, _PU32]),
    "polydet_plan_nodes": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_int32)]),
    "polydet_eval": (_I, [_VP, _VP, _I, _I, _VP, _VP, _VP]),
    "polydet_condense_batch": (_I, [_VP, _VP, _I, _I, _VP, _VP]),
    "polydet_interp": (_I, [_VP, _VP, _I, _I, _VP, _VP, _VP]),
    "polydet_interp_static": (_I, [_VP, _VP, _I, _I, _VP, _VP]),
    "polydet_crt": (_I, [_VP, _VP, _VP, _VP]),
    "polydet_crt_check": (_I, [_VP, _VP, _VP, _I, _VP, _VP]),
    "polydet_sync_status": (_I, [_VP, _VP, _PU32]),
    "polydet_batch_plan": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(Job), _I, _U32]),
    "polydet_batch_destroy": (_I, [_VP]),
    "polydet_batch_query": (_I, [_VP, ctypes.POINTER(BatchInfo)]),
    "polydet_batch_offsets": (_I, [_VP, _I, _PI64]),
    "polydet_batch_job_plan": (_I, [_VP, _I, ctypes.POINTER(_VP)]),
    "polydet_batch_set_launch": (_I, [_VP, _I, _I]),
    "polydet_batch_set_mode": (_I, [_VP, _I, _I]),
    "polydet_batch_set_chunk_words": (_I, [_VP, ctypes.c_uint64]),
    "polydet_batch_set_condense_ctas": (_I, [_VP, _I]),
    "polydet_team_size": (_I, [_I]),
    "polydet_batch_test_drop_copies": (_I, [_VP, _I]),
    "polydet_batch_eval": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "polydet_batch_eval_n": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "polydet_batch_condense": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "polydet_batch_condense_n": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "polydet_batch_interp": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "polydet_batch_crt": (_I, [_VP, _VP, _VP, _VP]),
    "polydet_batch_sync_status": (_I, [_VP, _VP, _PU32]),
    "polydet_mlp_forward": (_I, [_VP, _VP, _I, _VP, _VP, _VP]),
    "polydet_mlp_backward": (_I, [_VP, _VP, _VP, _I, _VP, _VP, _VP, _VP, _VP, _VP]),
    "polydet_mlp_adam": (_I, [_VP, _VP, _VP, _VP, _I, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, ctypes.c_float, _VP]),
    "polydet_probe_int_peaks": (_I, [_VP, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "polydet_condense_steps": (_I, [_I]),
    "polydet_last_error": (ctypes.c_char_p, []),
}


def lib():
    """Load libpolydet.so (raises if it is missing: no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpolydet.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    if _lib is None:
        return ""
    s = _lib.polydet_last_error()
    return s.decode() if s else ""


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise PolydetError(rc, what)


def prime_table() -> List[int]:
    L = lib()
    n = L.polydet_prime_table(None)
    buf = (ctypes.c_uint32 * n)()
    L.polydet_prime_table(buf)
    return list(buf)


def hadamard_primes(entry_l1: np.ndarray) -> tuple[int, float]:
    """Prime count and log2 of the coefficient bound from [n][n] l1 norms."""
    l1 = np.ascontiguousarray(entry_l1, dtype=np.int64)
    n = l1.shape[0]
    P = ctypes.c_int(0)
    lb = ctypes.c_double(0)
    _check(lib().polydet_hadamard_primes(n, l1.ctypes.data_as(_PI64), ctypes.byref(P),
                                         ctypes.byref(lb)), "polydet_hadamard_primes")
    return P.value, lb.value


def det_degree_bound(entry_degs, k: Optional[int] = None) -> tuple:
    """Per-variable degree bound of det(A) from the entries' degrees:
    ``entry_degs`` [n][n] of per-variable degree tuples, or None for a zero
    entry (the library's assignment bound, host only); ``k`` variables
    (taken from the entries when not given)."""
    n = len(entry_degs)
    if k is None:
        k = next((len(e) for r in entry_degs for e in r if e is not None), 1)
    arr = np.full((n, n, k), -1, dtype=np.int32)
    for i, r in enumerate(entry_degs):
        for j, e in enumerate(r):
            if e is not None:
                arr[i, j] = e
    out = (ctypes.c_int32 * k)()
    _check(lib().polydet_det_degree_bound(n, k, arr.ctypes.data_as(_PI32), out),
           "polydet_det_degree_bound")
    return tuple(out)


def entry_degrees(coeffs: np.ndarray, degs: Sequence[int]):
    """[n][n] per-variable degrees of the entries of a dense lex coefficient
    array [n][n][E] (None for a zero entry): input marshalling for
    det_degree_bound."""
    c = np.asarray(coeffs)
    n = c.shape[0]
    shape = tuple(int(d) + 1 for d in degs)
    out = []
    for i in range(n):
        row = []
        for j in range(n):
            t = c[i, j].reshape(shape)
            if not t.any():
                row.append(None)
                continue
            nz = np.nonzero(t)
            row.append(tuple(int(ax.max()) for ax in nz))
        out.append(row)
    return out


def unique_entries(coeffs: np.ndarray):
    """(map [n*n] int32, U, distinct coefficient rows [U][E]) of a dense
    coefficient array [n][n][E] (host only; -1 marks a zero entry)."""
    c = np.ascontiguousarray(coeffs, dtype=np.int32)
    n, E = c.shape[0], c.shape[2]
    m = np.empty(n * n, dtype=np.int32)
    U = ctypes.c_int32(0)
    uniq = np.empty((n * n, E), dtype=np.int32)
    _check(lib().polydet_unique_entries(n, E, c.ctypes.data_as(_PI32), m.ctypes.data_as(_PI32),
                                        ctypes.byref(U), uniq.ctypes.data_as(_PI32)),
           "polydet_unique_entries")
    return m, U.value, uniq[:U.value].copy()


def _ptr(t: torch.Tensor, dtype, numel: int, name: str) -> ctypes.c_void_p:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A polydet plan: n x n matrices in len(degs) variables, entry degree
    <= degs[v] in x_v, over the first ``nprimes`` primes of the table; node
    grid (default) or the paper's full power-of-two grid."""

    def __init__(self, n: int, degs: Sequence[int], nprimes: int, full_grid: bool = False,
                 det_degs: Optional[Sequence[int]] = None):
        L = lib()
        d = (ctypes.c_int32 * len(degs))(*[int(x) for x in degs])
        h = ctypes.c_void_p()
        flags = FLAG_FULL_GRID if full_grid else 0
        if det_degs is None:
            _check(L.polydet_plan(ctypes.byref(h), int(n), len(degs), d, int(nprimes), flags), "polydet_plan")
        else:
            D = (ctypes.c_int32 * len(degs))(*[int(x) for x in det_degs])
            _check(L.polydet_plan_degrees(ctypes.byref(h), int(n), len(degs), d, D, int(nprimes), flags),
                   "polydet_plan_degrees")
        self._h = h
        self._query()

    def _query(self) -> None:
        L = lib()
        h = self._h
        info = PlanInfo()
        _check(L.polydet_plan_query(h, ctypes.byref(info)), "polydet_plan_query")
        self.n, self.k, self.P, self.W = info.n, info.nvars, info.P, info.W
        self.E, self.G, self.C = info.E, info.G, info.C
        self.d = tuple(info.d[:self.k])
        self.D = tuple(info.D[:self.k])
        self.N = tuple(info.N[:self.k])
        self.M = tuple(info.M[:self.k])  # evaluation nodes per variable
        self.full_grid = bool(info.flags & FLAG_FULL_GRID)
        self.eval_ws_words = int(info.eval_ws_words)
        self.interp_ws_words = int(info.interp_ws_words)
        self.entries = int(info.entries)  # entries per prime of the evals tensor
        self.items = self.entries - 1 if info.unique >= 0 else self.entries  # evaluated entries
        pr = (ctypes.c_uint32 * self.P)()
        _check(L.polydet_plan_primes(h, pr), "polydet_plan_primes")
        self.primes = list(pr)
        rt = (ctypes.c_uint32 * (self.P * self.k))()
        _check(L.polydet_plan_roots(h, rt), "polydet_plan_roots")
        self.roots = [list(rt[q * self.k:(q + 1) * self.k]) for q in range(self.P)]
        self.node_exps = []  # node k of x_v is root_v ** node_exps[v][k]
        for v in range(self.k):
            ex = (ctypes.c_int32 * max(1, self.M[v]))()
            _check(L.polydet_plan_nodes(h, v, ex), "polydet_plan_nodes")
            self.node_exps.append(list(ex[:self.M[v]]))

    def set_entry_map(self, entry_map: np.ndarray, U: int) -> None:
        """Evaluate only the U distinct entries (map [n*n], -1 = zero entry):
        eval takes [U][E] coefficients and writes [prime][U + 1][G]."""
        m = np.ascontiguousarray(entry_map, dtype=np.int32)
        _check(lib().polydet_plan_set_entry_map(self._h, m.ctypes.data_as(_PI32), int(U)),
               "polydet_plan_set_entry_map")
        self._query()

    def stream_ws_words(self, rows: int = 1) -> int:
        """Workspace words eval_condense needs with slabs of ``rows`` nodes of x_1."""
        return int(lib().polydet_stream_ws_words(self._h, int(rows)))

    def eval_condense(self, coeffs: torch.Tensor, lo: int, hi: int, detvals: torch.Tensor,
                      ws: torch.Tensor, stream=None) -> None:
        """Evaluation and condensation streamed slab by slab through ``ws``."""
        _check(lib().polydet_eval_condense(
            self._h, _ptr(coeffs, torch.int32, self.items * self.E, "coeffs"), lo, hi,
            _ptr(detvals, torch.int32, (hi - lo) * self.G, "detvals"),
            _ptr(ws, torch.int32, 1, "workspace"), ctypes.c_uint64(ws.numel()), _stream(stream)),
            "polydet_eval_condense")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().polydet_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stages ------------------------------------------------------------
    def workspace(self, nprimes: int, device="cuda") -> torch.Tensor:
        """Scratch for eval/interp over ``nprimes`` primes at a time."""
        words = max(self.eval_ws_words, self.interp_ws_words, 1) * nprimes
        return torch.empty(words, dtype=torch.int32, device=device)

    def _ws(self, ws: Optional[torch.Tensor], per_prime: int, np_: int, what: str):
        if per_prime == 0:
            return ctypes.c_void_p(ws.data_ptr() if ws is not None else 0)
        if ws is None:
            raise ValueError(f"{what} needs a workspace of {per_prime} words per prime")
        return _ptr(ws, torch.int32, per_prime * np_, "workspace")

    def eval(self, coeffs: torch.Tensor, lo: int, hi: int, evals: torch.Tensor,
             ws: Optional[torch.Tensor] = None, stream=None) -> None:
        _check(lib().polydet_eval(self._h, _ptr(coeffs, torch.int32, self.items * self.E, "coeffs"), lo, hi,
                                  _ptr(evals, torch.int32, (hi - lo) * self.entries * self.G, "evals"),
                                  self._ws(ws, self.eval_ws_words, hi - lo, "polydet_eval"),
                                  _stream(stream)), "polydet_eval")

    def condense(self, evals: torch.Tensor, lo: int, hi: int, detvals: torch.Tensor, stream=None) -> None:
        _check(lib().polydet_condense_batch(
            self._h, _ptr(evals, torch.int32, (hi - lo) * self.entries * self.G, "evals"), lo, hi,
            _ptr(detvals, torch.int32, (hi - lo) * self.G, "detvals"), _stream(stream)),
            "polydet_condense_batch")

    def interp(self, detvals: torch.Tensor, lo: int, hi: int, residues: torch.Tensor,
               ws: Optional[torch.Tensor] = None, stream=None) -> None:
        _check(lib().polydet_interp(
            self._h, _ptr(detvals, torch.int32, (hi - lo) * self.G, "detvals"), lo, hi,
            _ptr(residues, torch.int32, (hi - lo) * self.C, "residues"),
            self._ws(ws, self.interp_ws_words, hi - lo, "polydet_interp"), _stream(stream)),
            "polydet_interp")

    def interp_static(self, detvals: torch.Tensor, lo: int, hi: int, residues: torch.Tensor,
                      stream=None) -> None:
        """polydet_interp without a workspace: scratch from the library's
        fixed device array (for callers that cannot allocate)."""
        _check(lib().polydet_interp_static(
            self._h, _ptr(detvals, torch.int32, (hi - lo) * self.G, "detvals"), lo, hi,
            _ptr(residues, torch.int32, (hi - lo) * self.C, "residues"), _stream(stream)),
            "polydet_interp_static")

    def crt(self, residues: torch.Tensor, limbs: torch.Tensor, stream=None) -> None:
        _check(lib().polydet_crt(self._h, _ptr(residues, torch.int32, self.P * self.C, "residues"),
                                 _ptr(limbs, torch.int32, self.C * self.W, "limbs"), _stream(stream)),
               "polydet_crt")

    def crt_check(self, residues: torch.Tensor, digits: torch.Tensor, i: int, unstable: torch.Tensor,
                  stream=None) -> None:
        """Digit i of every coefficient; ORs 1 into ``unstable`` when the
        reconstruction from i primes is changed by prime i (early stop)."""
        _check(lib().polydet_crt_check(self._h, _ptr(residues, torch.int32, (i + 1) * self.C, "residues"),
                                       _ptr(digits, torch.int32, (i + 1) * self.C, "digits"), int(i),
                                       _ptr(unstable, torch.int32, 1, "unstable"), _stream(stream)),
               "polydet_crt_check")

    def sync_status(self, stream=None) -> int:
        st = ctypes.c_uint32(0)
        rc = lib().polydet_sync_status(self._h, _stream(stream), ctypes.byref(st))
        if rc not in (OK, EBOUND, ETIMEOUT):
            _check(rc, "polydet_sync_status")
        return st.value


def tail_entry_words(M) -> int:
    """Words per entry of a materialized chunk for node counts M (per
    variable): rows of the first variable padded to 32 words when they hold
    at least 1024 nodes (the library's layout of the chunk)."""
    B = 1
    for m in M[1:]:
        B *= int(m)
    Bs = -(-B // 32) * 32 if B >= 1024 else B
    return int(M[0]) * Bs


def team_size(n: int) -> int:
    """Lanes per determinant in the condensation kernels of order n (a pure
    host query of the library's table)."""
    t = lib().polydet_team_size(int(n))
    if t < 1:
        _check(t, "polydet_team_size")
    return t


class Batch:
    """A polydet batch: jobs of any shape, one fused run for all of them.
    ``jobs`` is a list of (n, degs, nprimes)."""

    def __init__(self, jobs: Sequence[tuple], full_grid: bool = False):
        L = lib()
        arr = (Job * len(jobs))()
        for i, (n, degs, P) in enumerate(jobs):
            arr[i].n, arr[i].nvars, arr[i].nprimes = int(n), len(degs), int(P)
            arr[i].flags = FLAG_FULL_GRID if full_grid else 0
            for v, dv in enumerate(degs):
                arr[i].d[v] = int(dv)
        h = ctypes.c_void_p()
        _check(L.polydet_batch_plan(ctypes.byref(h), arr, len(jobs), 0), "polydet_batch_plan")
        self._h = h
        self.njobs = len(jobs)
        self.refresh()
        self.offsets = {}
        for name, which in (("coeffs", OFF_COEFFS), ("partial", OFF_PARTIAL), ("detvals", OFF_DETVALS),
                            ("residues", OFF_RESIDUES), ("limbs", OFF_LIMBS)):
            out = (ctypes.c_int64 * (self.njobs + 1))()
            _check(L.polydet_batch_offsets(h, which, out), "polydet_batch_offsets")
            self.offsets[name] = list(out)
        self.job_info = []
        for j in range(self.njobs):
            ph = ctypes.c_void_p()
            _check(L.polydet_batch_job_plan(h, j, ctypes.byref(ph)), "polydet_batch_job_plan")
            info = PlanInfo()
            _check(L.polydet_plan_query(ph, ctypes.byref(info)), "polydet_plan_query")
            self.job_info.append(info)

    def refresh(self) -> None:
        info = BatchInfo()
        _check(lib().polydet_batch_query(self._h, ctypes.byref(info)), "polydet_batch_query")
        self.info = info
        self.words = {"coeffs": info.coeff_words, "partial": info.partial_words,
                      "detvals": info.detval_words, "residues": info.residue_words,
                      "limbs": info.limb_words, "workspace": int(info.workspace_words)}

    def orders(self) -> List[int]:
        return [n for n in range(1, MAX_N + 1) if self.info.items[n] > 0]

    def set_launch(self, n: int, threads: int) -> None:
        _check(lib().polydet_batch_set_launch(self._h, int(n), int(threads)), "polydet_batch_set_launch")
        self.refresh()

    def set_mode(self, n: int, mode: int) -> None:
        """BATCH_FUSED or BATCH_MATERIALIZED for order n; rerun eval after it
        (the partial tensor's content and the workspace size change)."""
        _check(lib().polydet_batch_set_mode(self._h, int(n), int(mode)), "polydet_batch_set_mode")
        self.refresh()

    def mode(self, n: int) -> int:
        return int(self.info.mode[n])

    def set_chunk_words(self, words: int) -> None:
        """Budget (words) of one materialized chunk; at least one prime."""
        _check(lib().polydet_batch_set_chunk_words(self._h, int(words)), "polydet_batch_set_chunk_words")
        self.refresh()

    def set_condense_ctas(self, ctas_per_sm: int) -> None:
        """Cap the materialized orders' condensation at this many CTAs per SM
        (0: no cap) so that the first-variable passes run beside it."""
        _check(lib().polydet_batch_set_condense_ctas(self._h, int(ctas_per_sm)),
               "polydet_batch_set_condense_ctas")

    def test_drop_copies(self, on: bool) -> None:
        """Failure-detection test hook: withhold the fused kernels' bulk
        copies so that their bounded waits run out (status TIMEOUT)."""
        _check(lib().polydet_batch_test_drop_copies(self._h, int(bool(on))),
               "polydet_batch_test_drop_copies")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().polydet_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _p(self, t, name):
        return _ptr(t, torch.int32, max(1, self.words[name]), name)

    def eval(self, coeffs, partial, ws, stream=None, n: int = 0):
        _check(lib().polydet_batch_eval_n(self._h, int(n), self._p(coeffs, "coeffs"),
                                          self._p(partial, "partial"), self._p(ws, "workspace"),
                                          _stream(stream)), "polydet_batch_eval")

    def condense(self, partial, detvals, ws, stream=None, n: int = 0):
        _check(lib().polydet_batch_condense_n(self._h, int(n), self._p(partial, "partial"),
                                              self._p(detvals, "detvals"), self._p(ws, "workspace"),
                                              _stream(stream)), "polydet_batch_condense")

    def interp(self, detvals, residues, ws, stream=None):
        _check(lib().polydet_batch_interp(self._h, self._p(detvals, "detvals"),
                                          self._p(residues, "residues"), self._p(ws, "workspace"),
                                          _stream(stream)), "polydet_batch_interp")

    def crt(self, residues, limbs, stream=None):
        _check(lib().polydet_batch_crt(self._h, self._p(residues, "residues"), self._p(limbs, "limbs"),
                                       _stream(stream)), "polydet_batch_crt")

    def sync_status(self, stream=None) -> int:
        st = ctypes.c_uint32(0)
        rc = lib().polydet_batch_sync_status(self._h, _stream(stream), ctypes.byref(st))
        if rc not in (OK, EBOUND, ETIMEOUT):
            _check(rc, "polydet_batch_sync_status")
        return st.value


MLP_PARAMS = 4866


def _fptr(t: torch.Tensor, numel: int, name: str) -> ctypes.c_void_p:
    return _ptr(t, torch.float32, numel, name)


def mlp_forward(params, x, y, act=None, stream=None) -> None:
    B = x.shape[0]
    _check(lib().polydet_mlp_forward(_fptr(params, MLP_PARAMS, "params"), _fptr(x, B * 8, "x"), B,
                                     _fptr(y, B * 2, "y"),
                                     _fptr(act, B * 128, "act") if act is not None else None,
                                     _stream(stream)), "polydet_mlp_forward")


def mlp_backward(params, x, target, y, act, delta, grads, loss=None, stream=None) -> None:
    B = x.shape[0]
    _check(lib().polydet_mlp_backward(
        _fptr(params, MLP_PARAMS, "params"), _fptr(x, B * 8, "x"), _fptr(target, B * 2, "target"), B,
        _fptr(y, B * 2, "y"), _fptr(act, B * 128, "act"), _fptr(delta, B * 130, "delta"),
        _fptr(grads, MLP_PARAMS, "grads"), _fptr(loss, 1, "loss") if loss is not None else None,
        _stream(stream)), "polydet_mlp_backward")


def mlp_adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0,
             stream=None) -> None:
    _check(lib().polydet_mlp_adam(_fptr(params, MLP_PARAMS, "params"), _fptr(grads, MLP_PARAMS, "grads"),
                                  _fptr(m, MLP_PARAMS, "m"), _fptr(v, MLP_PARAMS, "v"), int(step),
                                  float(lr), float(beta1), float(beta2), float(eps),
                                  float(weight_decay), _stream(stream)), "polydet_mlp_adam")


def probe_int_peaks(stream=None) -> tuple[float, float, float, float]:
    """(32-bit multiply-adds per second, single-step modular updates per
    second, two-step element updates per second, three-step element updates
    per second) measured on the current device by the library's probes."""
    a = ctypes.c_double(0)
    u = ctypes.c_double(0)
    u2 = ctypes.c_double(0)
    u3 = ctypes.c_double(0)
    _check(lib().polydet_probe_int_peaks(_stream(stream), ctypes.byref(a), ctypes.byref(u), ctypes.byref(u2),
                                         ctypes.byref(u3)), "polydet_probe_int_peaks")
    return a.value, u.value, u2.value, u3.value


def condense_steps(n: int) -> int:
    """Elimination steps per pass of the condensation kernels of order n."""
    t = lib().polydet_condense_steps(int(n))
    if t < 1:
        _check(t, "polydet_condense_steps")
    return t


def limbs_to_ints(limbs: np.ndarray, W: int) -> List[int]:
    """[C][W] little-endian two's-complement uint32 words -> Python ints."""
    raw = np.ascontiguousarray(limbs, dtype=np.uint32).reshape(-1, W).astype("<u4").tobytes()
    step = 4 * W
    return [int.from_bytes(raw[i:i + step], "little", signed=True) for i in range(0, len(raw), step)]


def as_u32(t: torch.Tensor) -> np.ndarray:
    """Host copy of an int32 device tensor, reinterpreted as uint32."""
    return t.detach().cpu().numpy().view(np.uint32)
