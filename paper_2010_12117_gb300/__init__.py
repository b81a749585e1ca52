"""GB300-native exact determinants of polynomial matrices over Z[x1..xk].

The modular method of arXiv 2010.12117 (Algorithm 1): evaluate every entry on
a grid of roots of unity modulo many 31-bit NTT primes, take the determinant
of every evaluated matrix mod p, interpolate back, and reconstruct the signed
integer coefficients with Garner's mixed-radix CRT.  All four stages run in
hand-written sm_103a CUDA kernels behind the C-ABI library ``libpolydet``
(``include/polydet.h``); ``binding`` is its thin ctypes layer.

Submodules are imported lazily so that ``synth`` (seeded inputs) can be used
without the CUDA library.
"""
