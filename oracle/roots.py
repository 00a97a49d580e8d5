"""All complex roots of p to 60 digits (oracle; test infrastructure).

The paper treats root finding as a black box that returns the roots "to the
desired accuracy" (Section 2).  The oracle's black box is deliberately a
different algorithm from the CUDA path's Aberth iteration: companion-matrix
eigenvalues (numpy) as starting points, then Newton's method in mpmath at
``dps + 20`` digits.  The result is accepted only if every root has a tiny
relative residual, the roots are pairwise distinct and Vieta's first identity
holds; otherwise mpmath's own ``polyroots`` is used instead.
"""
from __future__ import annotations

import mpmath
import numpy as np

from .zpoly import trim


def _rel_residual(p, z):
    acc = mpmath.mpc(0)
    mag = mpmath.mpf(0)
    az = abs(z)
    for c in reversed(p):
        acc = acc * z + c
        mag = mag * az + abs(c)
    return abs(acc) / mag if mag else abs(acc)


def _newton(p, dp, z, tol, maxit=200):
    for _ in range(maxit):
        f = mpmath.mpc(0)
        for c in reversed(p):
            f = f * z + c
        g = mpmath.mpc(0)
        for c in reversed(dp):
            g = g * z + c
        if g == 0:
            return z, False
        step = f / g
        z = z - step
        if abs(step) <= tol * max(1, abs(z)):
            return z, True
    return z, False


def _checks(p, roots, dps):
    d = len(p) - 1
    lim = mpmath.mpf(10) ** (-(dps - 20))
    if len(roots) != d:
        return False
    if any(_rel_residual(p, z) > lim for z in roots):
        return False
    if abs(mpmath.fsum(roots) + p[-2]) > mpmath.mpf(10) ** (-(dps - 30)):
        return False
    sep = mpmath.mpf(10) ** (-(dps // 3))
    for i in range(d):
        for j in range(i + 1, d):
            if abs(roots[i] - roots[j]) < sep:
                return False
    return True


def complex_roots(p, dps: int = 60):
    """Return the d complex roots of the monic p as mpmath mpc values.

    The working precision is set to ``dps + 20`` digits inside; the returned
    values carry that precision."""
    p = trim(p)
    d = len(p) - 1
    if p[-1] != 1:
        raise ValueError("p must be monic")
    with mpmath.workdps(dps + 20):
        if d == 1:
            return [mpmath.mpc(-p[0])]
        dp = [i * p[i] for i in range(1, len(p))]
        start = np.roots(np.array([float(c) for c in reversed(p)], dtype=np.float64))
        tol = mpmath.mpf(10) ** (-(dps + 10))
        roots = []
        ok = len(start) == d
        for s in start:
            z, conv = _newton(p, dp, mpmath.mpc(complex(s)), tol)
            ok = ok and conv
            roots.append(z)
        if not (ok and _checks(p, roots, dps)):
            roots = list(mpmath.polyroots([mpmath.mpf(c) for c in reversed(p)],
                                          maxsteps=400, extraprec=4 * dps))
            roots = [mpmath.mpc(z) for z in roots]
            if not _checks(p, roots, dps):
                raise ArithmeticError("oracle root finder failed its own checks")
        return roots
