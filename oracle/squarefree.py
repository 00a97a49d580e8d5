"""Any nonzero p in Z[x]: the reductions of Section 2 (the paper names them:
a non-monic polynomial is transformed to a monic one, and Yun's algorithm
splits off the square-free parts), written plainly over Q with Python
Fractions.  Test infrastructure: only tests, the smoke check and the bench's
CPU baseline use this package.

  content(p)            p = content * pp, pp primitive with a positive
                        leading coefficient
  yun(pp)               Yun's square-free decomposition pp = prod a_i^i, each
                        a_i primitive, square-free, pairwise coprime
  factor_general(p)     content, then for every a_i: the monic transform
                        q(y) = lc^(e-1) a_i(y / lc), the oracle's factor() of
                        q, and the primitive part of g(lc x) for every monic
                        factor g of q, with multiplicity i
"""
from __future__ import annotations

from fractions import Fraction
from math import gcd
from typing import List, Tuple

from .factor import factor
from .zpoly import pmul, trim


def _qtrim(p):
    p = list(p)
    while len(p) > 1 and p[-1] == 0:
        p.pop()
    return p


def _qdivmod(a, b):
    """a = q b + r over Q, deg r < deg b."""
    a = [Fraction(c) for c in _qtrim(a)]
    b = [Fraction(c) for c in _qtrim(b)]
    if len(a) < len(b):
        return [Fraction(0)], a
    q = [Fraction(0)] * (len(a) - len(b) + 1)
    for k in range(len(a) - len(b), -1, -1):
        c = a[k + len(b) - 1] / b[-1]
        q[k] = c
        for j in range(len(b)):
            a[k + j] -= c * b[j]
    r = _qtrim(a[:len(b) - 1] or [Fraction(0)])
    return _qtrim(q), r


def _qgcd(a, b):
    """Monic gcd over Q by Euclid."""
    a, b = _qtrim([Fraction(c) for c in a]), _qtrim([Fraction(c) for c in b])
    while not (len(b) == 1 and b[0] == 0):
        a, b = b, _qdivmod(a, b)[1]
    return [c / a[-1] for c in a]


def _qderiv(p):
    return _qtrim([k * p[k] for k in range(1, len(p))] or [Fraction(0)])


def _qsub(a, b):
    n = max(len(a), len(b))
    return _qtrim([(a[k] if k < len(a) else 0) - (b[k] if k < len(b) else 0) for k in range(n)])


def _to_primitive_int(p):
    """A rational polynomial scaled to a primitive integer one with a
    positive leading coefficient."""
    den = 1
    for c in p:
        den = den * Fraction(c).denominator // gcd(den, Fraction(c).denominator)
    ints = [int(Fraction(c) * den) for c in p]
    g = 0
    for c in ints:
        g = gcd(g, c)
    if ints[-1] < 0:
        g = -g
    return trim([c // g for c in ints])


def content(p) -> Tuple[int, List[int]]:
    """p = c * pp with pp primitive and lc(pp) > 0."""
    p = trim(p)
    if p == [0]:
        raise ValueError("the zero polynomial")
    g = 0
    for c in p:
        g = gcd(g, c)
    if p[-1] < 0:
        g = -g
    return g, [c // g for c in p]


def yun(pp) -> List[Tuple[List[int], int]]:
    """Yun's algorithm over Q: [(a_i, i)] for the a_i of degree >= 1, with
    pp = prod a_i^i (each a_i primitive, lc > 0).  Steps: g = gcd(f, f'),
    b = f / g, c = f' / g, d = c - b'; then repeatedly a = gcd(b, d),
    b = b / a, c = d / a, d = c - b', until b is constant."""
    f = [Fraction(c) for c in trim(pp)]
    if len(f) == 1:
        return []
    fp = _qderiv(f)
    g = _qgcd(f, fp)
    b = _qdivmod(f, g)[0]
    c = _qdivmod(fp, g)[0]
    d = _qsub(c, _qderiv(b))
    out, i = [], 1
    while len(b) > 1:
        a = _qgcd(b, d)
        if len(a) > 1:
            out.append((_to_primitive_int(a), i))
        b = _qdivmod(b, a)[0]
        c = _qdivmod(d, a)[0]
        d = _qsub(c, _qderiv(b))
        i += 1
    return out


def _monic_transform(a):
    """q(y) = lc^(e-1) a(y / lc): q_k = a_k lc^(e-1-k), q_e = 1."""
    e, lc = len(a) - 1, a[-1]
    return [a[k] * lc ** (e - 1 - k) for k in range(e)] + [1]


def _back_transform(g, lc):
    """Primitive part of g(lc x)."""
    return _to_primitive_int([g[k] * lc ** k for k in range(len(g))])


def factor_general(p) -> Tuple[int, List[Tuple[List[int], int]]]:
    """(content, [(f, m), ...]) with p = content * prod f^m, every f
    irreducible over Z, primitive, lc > 0, in canonical order (degree, then
    coefficients a_0 .. a_e, then m)."""
    c, pp = content(p)
    out = []
    for a, i in yun(pp):
        lc = a[-1]
        q = _monic_transform(a)
        for g in factor(q).factors:
            out.append((_back_transform(g, lc), i))
    out.sort(key=lambda fm: (len(fm[0]) - 1, tuple(fm[0]), fm[1]))
    return c, out


def expand(c, factors):
    """c * prod f^m."""
    acc = [c]
    for f, m in factors:
        for _ in range(m):
            acc = pmul(acc, f)
    return trim(acc)
