"""The reduction of Section 2: real factorisation (Eq. 1), traces, rho (oracle).

Every root of p is either real (u_i) or one of a conjugate pair (z_j, conj
z_j).  Each real linear factor and each real quadratic factor of Eq. 1 is one
*element*.  For element k:

* ``t1`` is its contribution to the first trace Tr_1 (Eq. 4): u, or z+conj z;
* ``t2`` its contribution to the second trace Tr_2 (sum of squared roots):
  u^2, or z^2 + conj(z)^2;
* ``rho`` = frac(t1) with frac(x) = x - floor(x) (Section 2).

Order of elements (a reading; the paper indexes rho by "real roots first,
then complex pairs" and does not fix an order within each group): real roots
ascending, then pairs by (Re z, Im z) of the member with Im z > 0.  The
number of real roots r comes from the exact Sturm count and decides which
roots are real: the r roots of smallest |Im z|.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import mpmath

from .roots import complex_roots
from .sturm import real_root_count


@dataclass
class Element:
    kind: str            # "real" or "pair"
    root: object         # mpf (real) or mpc with Im > 0 (pair)
    degree: int          # 1 or 2
    t1: object           # mpf
    t2: object           # mpf
    rho: object          # mpf in [0, 1)


def frac(x):
    return x - mpmath.floor(x)


def elements_from_roots(roots, r: int, dps: int = 60) -> List[Element]:
    d = len(roots)
    if (d - r) % 2:
        raise ArithmeticError("real-root count has the wrong parity")
    with mpmath.workdps(dps + 20):
        by_im = sorted(roots, key=lambda z: abs(mpmath.im(z)))
        real = by_im[:r]
        cplx = by_im[r:]
        tiny = mpmath.mpf(10) ** (-(dps - 15))
        if any(abs(mpmath.im(z)) > tiny for z in real):
            raise ArithmeticError("a root counted real by Sturm has a non-negligible imaginary part")
        if any(abs(mpmath.im(z)) <= tiny for z in cplx):
            raise ArithmeticError("a non-real root has a negligible imaginary part")
        upper = sorted([z for z in cplx if mpmath.im(z) > 0], key=lambda z: (mpmath.re(z), mpmath.im(z)))
        lower = [z for z in cplx if mpmath.im(z) < 0]
        if len(upper) != len(lower):
            raise ArithmeticError("complex roots do not pair up")
        for z in upper:
            partner = min(lower, key=lambda w: abs(w - mpmath.conj(z)))
            if abs(partner - mpmath.conj(z)) > tiny:
                raise ArithmeticError("complex root without its conjugate")
        out = []
        for u in sorted(mpmath.re(z) for z in real):
            out.append(Element("real", u, 1, u, u * u, frac(u)))
        for z in upper:
            t1 = 2 * mpmath.re(z)
            t2 = 2 * mpmath.re(z * z)
            out.append(Element("pair", z, 2, t1, t2, frac(t1)))
        return out


def reduce_poly(p, dps: int = 60):
    """(roots, r, elements) for the monic square-free p."""
    roots = complex_roots(p, dps)
    r = real_root_count(p)
    return roots, r, elements_from_roots(roots, r, dps)
