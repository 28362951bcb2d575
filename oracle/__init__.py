"""Plain FP64 CPU oracle of the block-sparse sign-matrix path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs import it; the library never does.
It shares no code with the CUDA library: its arithmetic lives in
``bsr_oracle.c`` (plain loops, compiled with -ffp-contract=off) and ``sign.py``.

Parity pins (tests/test_oracle_*.py): dense numpy products on small inputs, the
dense eigendecomposition sign, closed forms (2x2, diagonal, block-diagonal),
the scalar Newton-Schulz recurrence on the eigenvalues, and the invariants
X^2 = 1, P^2 = P, Tr(P) = N_occ, PH = HP.
"""
