"""Exact polynomial arithmetic over Z and over F_l (oracle; test infrastructure).

Polynomials are lists of Python ints, ascending powers.  The zero polynomial
is ``[0]``.  Nothing here is approximate.
"""
from __future__ import annotations

from fractions import Fraction
from math import gcd
from typing import List, Tuple

Poly = List[int]

__all__ = ["trim", "deg", "padd", "psub", "pmul", "pscale", "pdivmod_monic",
           "pderiv", "peval", "content", "primitive", "prem", "gcd_mod",
           "is_squarefree", "is_monic", "SMALL_PRIMES"]


def trim(p) -> Poly:
    p = [int(c) for c in p]
    while len(p) > 1 and p[-1] == 0:
        p.pop()
    return p or [0]


def deg(p) -> int:
    p = trim(p)
    return -1 if p == [0] else len(p) - 1


def is_monic(p) -> bool:
    p = trim(p)
    return len(p) >= 2 and p[-1] == 1


def padd(a, b) -> Poly:
    n = max(len(a), len(b))
    return trim([(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)])


def psub(a, b) -> Poly:
    n = max(len(a), len(b))
    return trim([(a[i] if i < len(a) else 0) - (b[i] if i < len(b) else 0) for i in range(n)])


def pscale(a, c) -> Poly:
    return trim([c * x for x in a])


def pmul(a, b) -> Poly:
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return trim(out)


def pdivmod_monic(a, b) -> Tuple[Poly, Poly]:
    """Exact division of a by the monic b over Z: a = q*b + r, deg r < deg b."""
    a = trim(a)
    b = trim(b)
    if b[-1] != 1:
        raise ValueError("divisor must be monic")
    db = len(b) - 1
    if len(a) - 1 < db:
        return [0], a
    r = list(a)
    q = [0] * (len(a) - db)
    for k in range(len(a) - 1 - db, -1, -1):
        c = r[k + db]
        q[k] = c
        if c:
            for j in range(db + 1):
                r[k + j] -= c * b[j]
    return trim(q), trim(r[:db] if db > 0 else [0])


def pderiv(p) -> Poly:
    return trim([i * p[i] for i in range(1, len(p))] or [0])


def peval(p, x):
    acc = 0
    for c in reversed(p):
        acc = acc * x + c
    return acc


def content(p) -> int:
    g = 0
    for c in p:
        g = gcd(g, c)
    return g


def primitive(p) -> Poly:
    """p divided by its (positive) content."""
    g = content(p)
    return trim([c // g for c in p]) if g > 1 else trim(p)


def prem(a, b) -> Poly:
    """Pseudo-remainder: lc(b)^(deg a - deg b + 1) * a  mod  b, exact over Z."""
    a = trim(a)
    b = trim(b)
    da, db = len(a) - 1, len(b) - 1
    if da < db:
        return a
    lc = b[-1]
    r = list(a)
    for k in range(da - db, -1, -1):
        c = r[k + db]
        r = [lc * x for x in r]
        for j in range(db + 1):
            r[k + j] -= c * b[j]
    # r now carries lc^(da-db+1) * a - (...) * b with deg < db
    return trim(r[:db] if db > 0 else [0])


def _mod(p, ell) -> Poly:
    out = [c % ell for c in p]
    while len(out) > 1 and out[-1] == 0:
        out.pop()
    return out or [0]


def gcd_mod(a, b, ell) -> Poly:
    """Monic gcd of a and b over F_ell (ell prime), by Euclid."""
    a = _mod(a, ell)
    b = _mod(b, ell)
    while b != [0]:
        inv = pow(b[-1], ell - 2, ell)
        db = len(b) - 1
        r = list(a)
        while len(r) - 1 >= db and r != [0]:
            c = (r[-1] * inv) % ell
            shift = len(r) - 1 - db
            for j in range(db + 1):
                r[shift + j] = (r[shift + j] - c * b[j]) % ell
            while len(r) > 1 and r[-1] == 0:
                r.pop()
            if len(r) - 1 < db:
                break
        a, b = b, (r or [0])
    inv = pow(a[-1], ell - 2, ell)
    return [(c * inv) % ell for c in a]


SMALL_PRIMES = [p for p in range(3, 4000) if all(p % q for q in range(2, int(p ** 0.5) + 1))]


def _gcd_rational(a, b):
    a = [Fraction(c) for c in trim(a)]
    b = [Fraction(c) for c in trim(b)]
    def tr(p):
        while len(p) > 1 and p[-1] == 0:
            p.pop()
        return p
    a, b = tr(a), tr(b)
    while not (len(b) == 1 and b[0] == 0):
        r = list(a)
        while len(r) >= len(b) and not (len(r) == 1 and r[0] == 0):
            c = r[-1] / b[-1]
            shift = len(r) - len(b)
            for j in range(len(b)):
                r[shift + j] -= c * b[j]
            r.pop()
            r = tr(r) if r else [Fraction(0)]
        a, b = b, r
    return a


def is_squarefree(p) -> bool:
    """True iff gcd(p, p') = 1 over Q.  A prime ell with deg(p mod ell) =
    deg p and gcd(p mod ell, p' mod ell) = 1 certifies it; otherwise the
    exact rational Euclid decides."""
    p = trim(p)
    if deg(p) <= 1:
        return True
    dp = pderiv(p)
    for ell in SMALL_PRIMES[20:40]:
        if p[-1] % ell == 0:
            continue
        if len(gcd_mod(p, dp, ell)) == 1:
            return True
    return len(_gcd_rational(p, dp)) == 1
