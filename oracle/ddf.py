"""Irreducibility certificates by distinct-degree factorisation mod primes
(oracle; test infrastructure).

Not part of the paper's method: it is how the oracle knows the answer when
n is too large for the exhaustive scan (degree 100 and 120).  Textbook
facts used: if f in Z[x] is monic and square-free modulo a prime l, every
factor of f over Z reduces to a product of irreducible factors of f mod l, so
the degree of any factor over Z is a subset sum of the degrees of the
irreducible factors mod l.  Distinct-degree factorisation gives those
degrees: gcd(x^(l^k) - x, f) collects the irreducible factors of degree k.
Intersecting the achievable degree sets over several primes down to
{0, deg f} proves f irreducible.
"""
from __future__ import annotations

from collections import Counter

import numpy as np

from .zpoly import SMALL_PRIMES, gcd_mod, pderiv


def _trim(a):
    nz = np.nonzero(a)[0]
    return a[: nz[-1] + 1] if len(nz) else np.zeros(1, dtype=np.int64)


def _np(p, ell):
    return _trim(np.array([c % ell for c in p], dtype=np.int64))


def _rem(a, f, ell):
    """a mod f over F_ell, f monic (numpy int64, ascending)."""
    a = a.copy()
    df = len(f) - 1
    for k in range(len(a) - 1, df - 1, -1):
        c = a[k]
        if c:
            a[k - df:k + 1] = (a[k - df:k + 1] - c * f) % ell
    return _trim(a[:df]) if df > 0 else np.zeros(1, dtype=np.int64)


def _mulmod(a, b, f, ell):
    return _rem(np.convolve(a, b) % ell, f, ell)


def _powmod(base, e, f, ell):
    result = np.ones(1, dtype=np.int64)
    while e:
        if e & 1:
            result = _mulmod(result, base, f, ell)
        e >>= 1
        if e:
            base = _mulmod(base, base, f, ell)
    return result


def _exact_div_mod(a, b, ell):
    """a / b over F_ell (b divides a)."""
    a = [int(x) for x in a]
    b = [int(x) for x in b]
    inv = pow(b[-1], ell - 2, ell)
    q = [0] * (len(a) - len(b) + 1)
    for k in range(len(a) - len(b), -1, -1):
        c = (a[k + len(b) - 1] * inv) % ell
        q[k] = c
        for j in range(len(b)):
            a[k + j] = (a[k + j] - c * b[j]) % ell
    return q


def ddf_degrees(f, ell) -> Counter:
    """Degrees (with multiplicity) of the irreducible factors of f mod ell.
    f must be monic and square-free mod ell."""
    g = [int(x) for x in _np(f, ell)]
    k = 0
    h = np.array([0, 1], dtype=np.int64)
    out = Counter()
    while len(g) - 1 >= 2 * (k + 1):
        k += 1
        fn = np.array(g, dtype=np.int64)
        h = _powmod(_rem(h, fn, ell), ell, fn, ell)
        hx = [int(x) for x in h]
        hx += [0] * max(0, 2 - len(hx))
        hx[1] = (hx[1] - 1) % ell
        d = gcd_mod(hx, g, ell)
        if len(d) > 1:
            out[k] += (len(d) - 1) // k
            g = _exact_div_mod(g, d, ell)
    if len(g) > 1:
        out[len(g) - 1] += 1
    return out


def achievable_degrees(degs: Counter):
    sums = {0}
    for k, cnt in degs.items():
        for _ in range(cnt):
            sums = sums | {s + k for s in sums}
    return sums


def certify_irreducible(f, max_primes: int = 60):
    """(True, primes) if the degree sieve proves f irreducible over Z, else
    (False, primes tried)."""
    n = len(f) - 1
    if n <= 1:
        return True, []
    possible = set(range(n + 1))
    used = []
    df = pderiv(f)
    for ell in SMALL_PRIMES:
        if ell <= n:
            continue
        if len(gcd_mod(f, df, ell)) != 1:
            continue
        used.append(ell)
        possible &= achievable_degrees(ddf_degrees(f, ell))
        if possible == {0, n}:
            return True, used
        if len(used) >= max_primes:
            break
    return False, used
