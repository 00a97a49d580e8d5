"""Irreducible factors as atoms of the verified patterns (oracle).

Algorithm FACTOR returns every integer divisor it finds (Section 2).  The
irreducible factorisation is recovered from them: the root set of every
divisor is a union of root sets of irreducible factors, and each irreducible
factor's root set is itself a divisor, so with all divisors found the
minimal non-empty sets of the Boolean algebra they generate, atom(i) = the
intersection of every divisor set (or complement) that contains i, are
exactly the irreducible factors.
"""
from __future__ import annotations


def atoms(n: int, divisor_sets):
    full = frozenset(range(n))
    family = [full]
    for s in divisor_sets:
        s = frozenset(s)
        family.append(s)
        family.append(full - s)
    out = []
    seen = set()
    for i in range(n):
        a = full
        for t in family:
            if i in t:
                a = a & t
        if a not in seen:
            seen.add(a)
            out.append(a)
    return out
