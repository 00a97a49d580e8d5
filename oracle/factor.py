"""Algorithm FACTOR end to end (oracle; test infrastructure).

``factor(p)`` returns the canonical list of monic irreducible factors of the
monic square-free p.  With n (the number of real linear and quadratic
factors, Eq. 1) at most ``max_scan_n`` it runs the paper's pipeline in the
paper's order: roots, rho (Section 2), RECOMBINE_A (Section 3.1), the
"q in Z[x]" test of FACTOR, then the atoms of the verified divisors.  Above
that it cannot scan 2^(n-1) patterns; it then takes the known construction
(the factors a generator multiplied together), checks the product exactly and
certifies each factor irreducible by the distinct-degree sieve; a polynomial
with no construction is certified as a whole.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

from .atoms import atoms
from .ddf import certify_irreducible
from .recombine import ORACLE_M, fixed_point, recombine_a, window_for
from .reduction import reduce_poly
from .verify import integer_divisor
from .zpoly import is_monic, is_squarefree, pmul, trim


def canonical(factors):
    """Degree ascending, then (a_0, ..., a_{e-1}) lexicographic as signed ints."""
    return sorted((trim(f) for f in factors), key=lambda f: (len(f) - 1, tuple(f[:-1])))


@dataclass
class OracleResult:
    factors: List[List[int]]
    n: int = 0
    r: int = 0
    c: int = 0
    method: str = ""
    candidates: List[int] = field(default_factory=list)       # accepted s != 0 over the n-1 scanned elements
    verified: List[frozenset] = field(default_factory=list)   # element sets of the verified divisors
    certificate_primes: List[List[int]] = field(default_factory=list)
    elements: Optional[list] = None
    roots: Optional[list] = None


def _product(factors):
    acc = [1]
    for f in factors:
        acc = pmul(acc, f)
    return acc


def factor(p, construction=None, max_scan_n: int = 35, dps: int = 60) -> OracleResult:
    p = trim(p)
    if not is_monic(p):
        raise ValueError("p must be monic of degree >= 1")
    if not is_squarefree(p):
        raise ValueError("p must be square-free")
    d = len(p) - 1
    if d == 1:
        return OracleResult(factors=[p], n=1, r=1, c=0, method="trivial")
    roots, r, els = reduce_poly(p, dps)
    n = len(els)
    res = OracleResult(factors=[], n=n, r=r, c=(d - r) // 2, elements=els, roots=roots)
    if n <= max_scan_n:
        res.method = "exhaustive"
        w = fixed_point([e.rho for e in els])
        res.candidates = [s for s in recombine_a(w, ORACLE_M, window_for()) if s != 0]
        for s in res.candidates:
            subset = [i for i in range(n) if (s >> i) & 1]
            if integer_divisor(p, els, subset, dps) is not None:
                res.verified.append(frozenset(subset))
        facs = []
        for a in atoms(n, res.verified):
            q = integer_divisor(p, els, sorted(a), dps)
            if q is None:
                raise ArithmeticError("an atom of verified divisors is not an integer divisor")
            facs.append(q)
        res.factors = canonical(facs)
    else:
        res.method = "certificate"
        facs = []
        for f in (construction or [p]):
            f = trim(f)
            ok, primes = certify_irreducible(f)
            if ok:
                facs.append(f)
                res.certificate_primes.append(primes)
            elif f != p and len(f) - 1 < d:
                # a construction factor that is itself reducible: factor it
                # on its own (by scan when its n is small enough)
                sub = factor(f, None, max(max_scan_n, 35), dps)
                facs.extend(sub.factors)
                res.certificate_primes.extend(sub.certificate_primes)
            else:
                raise ArithmeticError("could not certify a factor irreducible; n too large to scan")
        res.factors = canonical(facs)
    if _product(res.factors) != p:
        raise ArithmeticError("product of factors differs from p")
    return res
