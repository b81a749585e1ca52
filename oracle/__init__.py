"""CPU oracle for the exact determinant of a polynomial matrix over Z[x1..xk].

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
and the CPU-baseline leg of the benchmark may import anything from here.  The
CUDA path never routes through it, and nothing here imports the CUDA path.

Everything is plain, slow, single-threaded Python on Python ints (exact), so
that each function can be read against the paper by eye:

* ``poly``        - dense/dict multivariate polynomials, the lex coefficient
                    encoding and degree padding of Sec. 2.
* ``bareiss``     - the determinant itself: fraction-free Bareiss elimination
                    over Z[x1..xk] (O1), integer Bareiss after Kronecker
                    packing (O2), and Leibniz brute force for tiny matrices.
* ``modular``     - the stage-by-stage references of Sec. 3: NTT primes
                    (Eq. 1), roots of unity, evaluation on the root grid
                    (Sec. 3.1), determinant mod p (Sec. 3.2), interpolation
                    (Sec. 3.3), mixed-radix / Garner reconstruction (Sec. 3.4).
* ``plan``        - degree bounds, grid sizes, the coefficient bound and the
                    prime count (Sec. 2).
* ``certificate`` - Schwartz-Zippel check for outputs too large for O1/O2.
* ``predict``     - the run-time prediction formula of Sec. 5.

Pins (tests marked ``not gpu``) tie each function to values the paper prints
or the mathematics fixes.  ``modular.count_ntt_primes_after`` is pinned by
hand-counted cases and an independent count; only its comparison with the
printed prime-count table of Sec. 4.2 is unpinned, because the paper's
counting rule cannot be recovered exactly.
"""
