"""Shared test helpers (host logic only; no method arithmetic)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def ensure_lib():
    """Build libpolydet.so if it is missing, then load it."""
    from paper_2010_12117_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.lib()


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def evals_tensor(mats: np.ndarray, G: int):
    """Host matrices [P][G][n][n] of residues -> the evals layout
    [P][n*n][G] as an int32 CUDA tensor."""
    import torch
    P, g, n, _ = mats.shape
    assert g == G
    arr = np.ascontiguousarray(mats.reshape(P, G, n * n).transpose(0, 2, 1)).astype(np.uint32)
    return torch.from_numpy(arr.view(np.int32).reshape(-1)).cuda()


def random_residue_mats(rng, P, G, n, primes, zero_frac=0.0):
    out = np.empty((P, G, n, n), dtype=np.uint64)
    for q in range(P):
        m = rng.integers(0, primes[q], (G, n, n), dtype=np.uint64)
        if zero_frac:
            m[rng.random((G, n, n)) < zero_frac] = 0
        out[q] = m
    return out


def oracle_check_member(args):
    """One GPU result checked by the oracle, in a worker process (no torch
    import): bit-exact against O2 when ``exact``, else the Schwartz-Zippel
    certificate with ``trials`` points.  Returns (kind, ok, seconds)."""
    import time
    from oracle import bareiss, certificate, plan
    coeffs, degs, got, exact, trials = args
    t = time.perf_counter()
    if exact:
        ok = bareiss.det_packed(coeffs, degs) == got
        kind = "exact"
    else:
        D = plan.det_degree_bound(len(coeffs), degs)
        ok = certificate.check(coeffs, degs, got, D, trials=trials)
        kind = "certified"
    return kind, ok, time.perf_counter() - t
