"""Run-time prediction of Sec. 5 (Eq. for T).

T = C_p * r^2 * Round(mean_i T_e_i, 2) * mu, where C_p is the number of
primes, r the order, T_e_i the FFT time of entry i over one prime, and
mu = (unique entries) / r^2 the replication factor.  Reading of the garbled
sum index: the mean runs over all r^2 entries.
"""
from __future__ import annotations

from typing import Sequence


def predict_seconds(num_primes: int, r: int, entry_times: Sequence[float],
                    unique_entries: int | None = None) -> float:
    mean = sum(entry_times) / len(entry_times)
    mu = (unique_entries if unique_entries is not None else r * r) / (r * r)
    return num_primes * r * r * round(mean, 2) * mu
