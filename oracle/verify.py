"""Candidate verification of Algorithm FACTOR (oracle; test infrastructure).

For a pattern (a subset of the elements of Eq. 1) the candidate factor is
q = prod (x - u_i) * prod (x^2 - (z_j + conj z_j) x + z_j conj z_j) (Eq. 2).
FACTOR keeps q iff q lies in Z[x] (Section 2).  The oracle multiplies q out at
the roots' working precision, requires every coefficient to be within
10^-(dps/3) of an integer, rounds, and then proves divisibility exactly:
p = q * h with zero remainder in Python integers.
"""
from __future__ import annotations

import mpmath

from .zpoly import pdivmod_monic, trim


def element_poly(el):
    if el.kind == "real":
        return [-el.root, mpmath.mpf(1)]
    z = el.root
    return [mpmath.re(z * mpmath.conj(z)), -2 * mpmath.re(z), mpmath.mpf(1)]


def real_product(elements, subset, dps: int = 60):
    with mpmath.workdps(dps + 20):
        q = [mpmath.mpf(1)]
        for k in subset:
            f = element_poly(elements[k])
            out = [mpmath.mpf(0)] * (len(q) + len(f) - 1)
            for i, a in enumerate(q):
                for j, b in enumerate(f):
                    out[i + j] += a * b
            q = out
        return q


def integer_divisor(p, elements, subset, dps: int = 60):
    """The integer polynomial of the pattern if it divides p, else None."""
    q = real_product(elements, subset, dps)
    with mpmath.workdps(dps + 20):
        tol = mpmath.mpf(10) ** (-(dps // 3))
        qi = []
        for c in q:
            k = int(mpmath.nint(c))
            if abs(c - k) > tol:
                return None
            qi.append(k)
    qi = trim(qi)
    _, rem = pdivmod_monic(p, qi)
    return qi if rem == [0] else None
