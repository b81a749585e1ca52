"""C ABI checks that need no GPU: the library loads, exports every function
declared in include/polydet.h, the binding covers them, and the host-only
planning calls agree with the oracle's independent versions."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from helpers import ROOT, ensure_lib
from oracle import modular, plan as oplan

HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(polydet_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = ensure_lib()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), f"{name} declared but not exported"
    from paper_2010_12117_gb300 import binding
    nm = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True)
    exported = set(re.findall(r"\bpolydet_[a-z0-9_]+\b", nm.stdout))
    assert set(names) <= exported


def test_binding_covers_the_header():
    from paper_2010_12117_gb300 import binding
    assert set(declared_functions()) <= set(binding.SIGNATURES)


def test_prime_table_matches_oracle():
    ensure_lib()
    from paper_2010_12117_gb300 import binding
    assert binding.prime_table() == modular.ntt_primes()


def _l1_from_bits(rng, n, bits):
    return rng.integers(0, 2 ** bits, (n, n), dtype=np.int64)


@pytest.mark.parametrize("n,bits", [(1, 5), (4, 8), (12, 20), (16, 30), (24, 22), (32, 25)])
def test_hadamard_prime_count_matches_oracle(n, bits):
    ensure_lib()
    from paper_2010_12117_gb300 import binding
    rng = np.random.default_rng(n * 100 + bits)
    for _ in range(5):
        l1 = _l1_from_bits(rng, n, bits)
        # an integer matrix with these l1 norms (constants) has the same bound
        coeffs = l1.reshape(n, n, 1).tolist()
        want = oplan.primes_needed(oplan.hadamard_bound_sq(coeffs, (0,)), modular.ntt_primes())
        got, _ = binding.hadamard_primes(l1)
        # the library works in floating point with a 1e-6-bit safety margin: it
        # may take one prime more than the exact rule, never fewer
        assert got in (want, want + 1)


def test_hadamard_zero_matrix_and_errors():
    ensure_lib()
    from paper_2010_12117_gb300 import binding
    P, lb = binding.hadamard_primes(np.zeros((3, 3), dtype=np.int64))
    assert P == 2
    L = binding.lib()
    out = ctypes.c_int(0)
    assert L.polydet_hadamard_primes(0, None, ctypes.byref(out), None) == binding.EINVAL


def test_team_sizes_are_usable_and_match_the_tuner():
    """Lanes per determinant: a power of two dividing every candidate CTA
    size, small enough that a lane holds at most 8 columns of a 32x32
    matrix; the tuner's candidate list follows the library's table."""
    ensure_lib()
    from paper_2010_12117_gb300 import binding, tune
    for n in range(1, 33):
        t = binding.team_size(n)
        assert t in (1, 2, 4, 8, 16), (n, t)
        assert -(-n // t) <= 16
        assert tune.team(n) == t
        assert all(th % t == 0 for mode, th in tune.candidates(n))
    with pytest.raises(binding.PolydetError):
        binding.team_size(0)
    with pytest.raises(binding.PolydetError):
        binding.team_size(33)


def test_condense_steps_cover_every_order():
    """The fast elimination takes two or three steps per pass at every order
    (Fast2Step / Fast3Step); orders outside 1..32 are rejected."""
    ensure_lib()
    from paper_2010_12117_gb300 import binding
    steps = [binding.condense_steps(n) for n in range(1, 33)]
    assert set(steps) <= {2, 3}, steps
    assert 3 in steps and 2 in steps
    for bad in (0, 33):
        with pytest.raises(binding.PolydetError):
            binding.condense_steps(bad)


def _rand_edeg(rng, n, k, dmax, pzero):
    return [[None if rng.random() < pzero else tuple(int(x) for x in rng.integers(0, dmax + 1, k))
             for _ in range(n)] for _ in range(n)]


@pytest.mark.parametrize("n", [1, 2, 4, 6, 9, 13, 20, 32])
def test_det_degree_bound_matches_oracle(n):
    """The library's assignment bound (Hungarian method) against the oracle's
    (brute force over permutations, or scipy's matching), with zero entries,
    including matrices whose zeros leave no permutation (bound 0)."""
    ensure_lib()
    from paper_2010_12117_gb300 import binding
    rng = np.random.default_rng(900 + n)
    for pz in (0.0, 0.3, 0.7):
        for _ in range(4):
            e = _rand_edeg(rng, n, 3, 12, pz)
            assert binding.det_degree_bound(e, 3) == oplan.assignment_degree_bound(e, 3), (n, pz)


def test_det_degree_bound_of_the_four_variable_sylvester_target():
    ensure_lib()
    from paper_2010_12117_gb300 import binding, synth
    pm = synth.sylvester_15_four_vars(0)
    e = binding.entry_degrees(pm.coeffs, pm.degs)
    assert binding.det_degree_bound(e) == (298, 171, 119, 45)
    assert oplan.assignment_degree_bound(e, 4) == (298, 171, 119, 45)


def test_unique_entries_against_an_independent_grouping():
    """Entries with equal coefficient vectors share an index, in order of
    first occurrence; zero entries map to -1; the distinct rows are the
    first occurrences."""
    ensure_lib()
    from paper_2010_12117_gb300 import binding, synth
    rng = np.random.default_rng(5)
    cases = [synth.sylvester_16(1).coeffs, synth.random_matrix(rng, 7, (2, 1), 0.5, -3, 3).coeffs,
             np.zeros((3, 3, 4), dtype=np.int64)]
    base = rng.integers(-9, 9, (4, 6))
    pick = rng.integers(0, 5, (6, 6))
    c = np.zeros((6, 6, 6), dtype=np.int64)
    for i in range(6):
        for j in range(6):
            c[i, j] = base[pick[i, j]] if pick[i, j] < 4 else 0
    cases.append(c)
    for coeffs in cases:
        n, E = coeffs.shape[0], coeffs.shape[2]
        m, U, uniq = binding.unique_entries(coeffs)
        flat = coeffs.reshape(n * n, E)
        seen = {}
        want = []
        for e in range(n * n):
            key = tuple(int(x) for x in flat[e])
            if not any(key):
                want.append(-1)
                continue
            if key not in seen:
                seen[key] = len(seen)
            want.append(seen[key])
        assert list(m) == want
        assert U == len(seen)
        for key, u in seen.items():
            assert tuple(int(x) for x in uniq[u]) == key
    m, U, _ = binding.unique_entries(synth.sylvester_16(1).coeffs)
    assert U == 18  # f_0..f_8 and g_0..g_8
