"""Number of real roots by an exact Sturm sequence (oracle; test infrastructure).

Textbook Sturm theorem: for square-free p with S_0 = p, S_1 = p' and
S_{k+1} = -rem(S_{k-1}, S_k), the number of distinct real roots equals
V(-inf) - V(+inf), V counting sign changes.  Each S_{k+1} is replaced by a
positive multiple of itself (pseudo-remainder with the sign of lc^(delta+1)
corrected, then divided by its positive content), which leaves every sign
unchanged and keeps the integers small.
"""
from __future__ import annotations

from .zpoly import deg, pderiv, prem, primitive, trim


def sturm_sequence(p):
    p = trim(p)
    seq = [p, pderiv(p)]
    while deg(seq[-1]) > 0:
        a, b = seq[-2], seq[-1]
        r = prem(a, b)
        k = deg(a) - deg(b) + 1
        if (b[-1] < 0) and (k % 2 == 1):
            r = [-c for c in r]              # now a positive multiple of rem(a, b)
        nxt = [-c for c in r]
        if deg(nxt) < 0:
            break
        seq.append(primitive(nxt))
    return seq


def _sign_changes(signs):
    s = [x for x in signs if x != 0]
    return sum(1 for i in range(1, len(s)) if s[i] != s[i - 1])


def real_root_count(p) -> int:
    """Distinct real roots of p (exact)."""
    seq = sturm_sequence(p)
    at_pos = [1 if q[-1] > 0 else -1 for q in seq if deg(q) >= 0]
    at_neg = [(1 if q[-1] > 0 else -1) * (-1 if deg(q) % 2 else 1) for q in seq if deg(q) >= 0]
    return _sign_changes(at_neg) - _sign_changes(at_pos)
