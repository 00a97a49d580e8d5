"""CPU oracle for the Real-Factors-Recombination (RFR) hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the paper's method computes, used to check the CUDA path.
Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import it; the library under ``paper_2410_15880_b300`` never does, and
this package imports nothing from the library (the two share no code; only the
seeded generators in ``workloads`` feed both).

What it computes (the plain definition): the complete factorisation of a
monic, square-free p in Z[x] into monic irreducible factors, in canonical
order (degree ascending, then a_0..a_{e-1} lexicographic as signed ints).
How (Section 2 and Section 3.1 of the paper, in their order):

* roots of p to 60 digits (``roots``), real count r from an exact Sturm
  sequence (``sturm``);
* the real factorisation of Eq. 1 and the vector rho of fractional parts of
  the first traces (``reduction``, Section 2);
* RECOMBINE_A, the exhaustive scan over 2^(n-1) patterns with value (Eq. 8)
  and accept (Eq. 9) (``recombine``, Section 3.1);
* the FACTOR test "q in Z[x]" by rounding and exact division (``verify``);
* the irreducible factors as atoms of the verified patterns (``atoms``);
* for n too large to scan, the known construction plus irreducibility
  certificates from distinct-degree factorisation modulo small primes
  (``ddf``).

Pins (tests marked ``not gpu``) tie each function to something other than
itself: brute-force divisor search on tiny inputs, cyclotomic closed forms,
the Swinnerton-Dyer polynomials of Eq. 5-7, known products, Vieta and Newton
identities, and the product-equals-input invariant.
"""
from .zpoly import *          # noqa: F401,F403
from .factor import factor, canonical, OracleResult   # noqa: F401
