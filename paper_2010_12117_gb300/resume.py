"""Stage-wise restart points (Sec. 4.3): per-prime determinant residues.

After interpolation the residues of one prime are the determinant mod that
prime; they are all a run needs to resume.  A ``ResidueStore`` keeps them as
one file per prime beside a manifest that records the job (order, degrees,
prime list, a digest of the input) and a SHA-256 of every file.  A file that
is missing, truncated or fails its checksum is treated as not computed, so a
resumed run recomputes exactly those primes.  Writes go to a temporary name
and are renamed into place, so a process killed mid-write leaves no partial
file under the final name.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, List, Optional, Sequence

import numpy as np


def input_digest(coeffs: np.ndarray, degs: Sequence[int]) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(coeffs, dtype=np.int64).tobytes())
    h.update(json.dumps([int(d) for d in degs]).encode())
    return h.hexdigest()


class ResidueStore:
    def __init__(self, path: str):
        self.path = path
        os.makedirs(path, exist_ok=True)
        self.manifest_path = os.path.join(path, "manifest.json")

    # -- manifest ----------------------------------------------------------
    def _read_manifest(self) -> Optional[dict]:
        try:
            with open(self.manifest_path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return None

    def _write_manifest(self, m: dict) -> None:
        tmp = self.manifest_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(m, f)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, self.manifest_path)

    def open_job(self, job: dict) -> dict:
        """Bind the store to a job; a manifest for a different job is reset."""
        m = self._read_manifest()
        if m is None or m.get("job") != job:
            m = {"job": job, "primes": {}}
            self._write_manifest(m)
        return m

    # -- per-prime residues -------------------------------------------------
    def _file(self, q: int) -> str:
        return os.path.join(self.path, f"residues_p{q:03d}.u32")

    def save(self, q: int, residues: np.ndarray) -> None:
        data = np.ascontiguousarray(residues, dtype=np.uint32).astype("<u4").tobytes()
        tmp = self._file(q) + ".tmp"
        with open(tmp, "wb") as f:
            f.write(data)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, self._file(q))
        m = self._read_manifest() or {"job": None, "primes": {}}
        m["primes"][str(q)] = {"sha256": hashlib.sha256(data).hexdigest(), "words": len(data) // 4}
        self._write_manifest(m)

    def load(self, q: int, words: int) -> Optional[np.ndarray]:
        m = self._read_manifest()
        if not m:
            return None
        ent = m["primes"].get(str(q))
        if not ent or ent["words"] != words:
            return None
        try:
            with open(self._file(q), "rb") as f:
                data = f.read()
        except OSError:
            return None
        if len(data) != 4 * words or hashlib.sha256(data).hexdigest() != ent["sha256"]:
            return None
        return np.frombuffer(data, dtype="<u4").astype(np.uint32)

    def done(self, P: int, words: int) -> Dict[int, np.ndarray]:
        out = {}
        for q in range(P):
            r = self.load(q, words)
            if r is not None:
                out[q] = r
        return out

    def missing(self, P: int, words: int) -> List[int]:
        have = self.done(P, words)
        return [q for q in range(P) if q not in have]
