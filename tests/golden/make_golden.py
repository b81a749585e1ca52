"""Write the stored expected values for workloads too slow for the oracle to
run inside the test suite.  Calls only the CPU oracle (``oracle/``) and the
seeded input generators; nothing here touches the CUDA path.

    python tests/golden/make_golden.py            # 12x12 over Z[x,y,z], seed 0 (about 10 min)

Each file records the SHA-256 of the full coefficient list (decimal, comma
separated, lex order over the box prod [0, D_v]), its length, the number of
nonzero coefficients, the largest bit length, and a seeded sample of
individual coefficients.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import bareiss, plan  # noqa: E402
from paper_2010_12117_gb300 import synth  # noqa: E402


def digest(coeffs) -> str:
    return hashlib.sha256(",".join(str(int(c)) for c in coeffs).encode()).hexdigest()


def write(name: str, seed: int, pm, out, seconds: float, oracle_name: str) -> str:
    D = plan.det_degree_bound(pm.n, pm.degs)
    rng = np.random.default_rng(2024)
    idx = sorted(set(int(i) for i in rng.integers(0, len(out), 96)) |
                 {0, len(out) - 1} |
                 set(int(i) for i in np.argsort([-abs(c) for c in out])[:16]))
    rec = {
        "workload": name, "seed": seed, "n": pm.n, "degs": list(pm.degs), "D": list(D),
        "coefficients": len(out), "nonzero": sum(1 for c in out if c),
        "max_bits": max(abs(c) for c in out).bit_length(),
        "sha256": digest(out),
        "samples": {str(i): str(out[i]) for i in idx},
        "oracle": oracle_name, "oracle_seconds": round(seconds, 1),
        "cmd": "python tests/golden/make_golden.py",
    }
    path = os.path.join(HERE, f"{name}_seed{seed}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    return path


def main() -> None:
    pm = synth.sparse_12x12_xyz(0)
    t = time.time()
    out = bareiss.det_packed(pm.coeffs.tolist(), pm.degs)
    print(write("sparse_12x12_xyz", 0, pm, out, time.time() - t, "O2 packed Bareiss"))


if __name__ == "__main__":
    main()
