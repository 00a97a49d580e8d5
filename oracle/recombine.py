"""RECOMBINE_A and the plain definitions behind the MITM stages (oracle).

Section 3.3 moves the search from rho in [0,1)^n to integer weights
w_i = rho_i * M in Z_M (Eq. 18) with value(s) = (sum_i s_i w_i) mod M.  The
oracle takes that step with two readings of the text:

* rounding instead of floor when forming w_i (Eq. 18 floors, so n floors
  could pile up n units of error while Eq. 19 still asks for exact 0 or M-1);
* a circular window: accept(y) iff min(y, M - y) <= window, which is Eq. 9
  (y < eps or 1 - y < eps) written in units of 1/M.

The oracle's own modulus is M = 2^62 and its window is eps = 1e-12: roots
correct to ~1e-40 put a true divisor within ~1e-38 of an integer, and a false
pattern lands inside the window with probability ~2e-12.
"""
from __future__ import annotations

import mpmath
import numpy as np

ORACLE_BITS = 62
ORACLE_M = 1 << ORACLE_BITS
ORACLE_EPS = 1e-12


def fixed_point(rhos, bits: int = ORACLE_BITS):
    """w_i = round(rho_i * 2^bits) mod 2^bits (Eq. 18, rounded)."""
    m = 1 << bits
    return [int(mpmath.nint(rho * m)) % m for rho in rhos]


def value(s: int, w, M: int) -> int:
    """Eq. 8 / Eq. 18: the sum of the weights selected by pattern s, mod M."""
    return sum(w[i] for i in range(len(w)) if (s >> i) & 1) % M


def accept(y: int, M: int, window: int) -> bool:
    """Eq. 9 / Eq. 19 with the circular window."""
    return y <= window or M - y <= window


def window_for(eps: float = ORACLE_EPS, M: int = ORACLE_M) -> int:
    return int(eps * M)


def recombine_a(w, M: int = ORACLE_M, window: int | None = None):
    """RECOMBINE_A (Section 3.1): every pattern s < 2^(n-1) whose value is
    accepted.  Complement symmetry (Section 3.1) keeps the last element out of
    every scanned pattern.  Includes the trivial pattern s = 0.

    Small n: a literal loop over s.  Larger n: the same value(s) for every s,
    evaluated as a vectorised sum over the pattern's bits (low bits by
    doubling a table, high bits added as a scalar per chunk)."""
    if window is None:
        window = window_for(M=M)
    n = len(w)
    if n == 0:
        return [0]
    nbits = n - 1
    if nbits <= 16:
        return [s for s in range(1 << nbits) if accept(value(s, w, M), M, window)]
    if M > (1 << 62) and M != (1 << 64):
        raise ValueError("vectorised scan needs M <= 2^62 or M = 2^64 (uint64 wrap-around)")
    mask = np.uint64(M - 1)
    low = min(nbits, 20)
    vals = np.zeros(1, dtype=np.uint64)
    for i in range(low):
        vals = np.concatenate([vals, (vals + np.uint64(w[i])) & mask])
    out = []
    win = np.uint64(window)
    top = np.uint64(M - window)
    for hi in range(1 << (nbits - low)):
        base = 0
        for j in range(nbits - low):
            if (hi >> j) & 1:
                base += w[low + j]
        y = (vals + np.uint64(base % M)) & mask
        idx = np.nonzero((y <= win) | (y >= top))[0]
        out.extend(int((hi << low) | int(k)) for k in idx)
    return out


def expand_values(w, M: int):
    """EXPAND (Section 3.3) before its sort: value(s) for s = 0 .. 2^h - 1, in
    pattern order."""
    return [value(s, w, M) for s in range(1 << len(w))]


def expand(w, M: int):
    """EXPAND: the sorted list of all half-subset values."""
    return sorted(expand_values(w, M))


def band_pairs(alpha_vals, beta_vals, M: int, window: int):
    """The set FIND is meant to produce, by brute force over all pairs: every
    (i, j) with accept(alpha_i + beta_j).  Reading of FIND: the acceptance is
    circular (sums near 0 as well as near M) and every pair in the window is
    reported, not only the first per i."""
    return {(i, j) for i, a in enumerate(alpha_vals) for j, b in enumerate(beta_vals)
            if accept((a + b) % M, M, window)}


def _signed64(x: int) -> int:
    x %= 1 << 64
    return x - (1 << 64) if x >= (1 << 63) else x


def expand_values_u64(w):
    """EXPAND (Section 3.3) before its sort, modulo 2^64, as a uint64 array in
    pattern order: entry s is the sum of w[i] over the set bits i of s.
    (Sums are formed on the int64 view: two's-complement addition is
    addition modulo 2^64.)"""
    vals = np.zeros(1, dtype=np.int64)
    for x in w:
        vals = np.concatenate([vals, vals + _signed64(int(x))])
    return vals.view(np.uint64)


def band_pairs_sorted(w_a, w_b, window: int):
    """The pair set of band_pairs for M = 2^64 and halves too large to pair
    by brute force: every (i, j) whose value alpha_i + beta_j (sums of the
    half-a weights over the bits of i and of the half-b weights over the bits
    of j) is accepted.  The meet in the middle of Section 3.3 written with a
    library sort: beta is sorted once and, for every alpha_i, the betas in
    the circular window [-alpha_i - window, -alpha_i + window] are found by
    binary search."""
    alpha = expand_values_u64(w_a)
    beta = expand_values_u64(w_b)
    if window >= (1 << 63):
        return {(i, j) for i in range(len(alpha)) for j in range(len(beta))}
    order = np.argsort(beta, kind="stable")
    sb = beta[order]
    neg = -alpha.view(np.int64)                           # -alpha_i modulo 2^64
    lo = (neg - _signed64(window)).view(np.uint64)
    hi = (neg + _signed64(window)).view(np.uint64)
    out = set()
    wrap = lo > hi                                        # the window runs over 2^64 -> 0
    a0 = np.searchsorted(sb, lo, side="left")
    a1 = np.searchsorted(sb, hi, side="right")
    for i in np.nonzero(~wrap & (a1 > a0))[0]:
        out.update((int(i), int(j)) for j in order[a0[i]:a1[i]])
    for i in np.nonzero(wrap)[0]:                         # [lo, 2^64) and [0, hi]
        out.update((int(i), int(j)) for j in order[:a1[i]])
        out.update((int(i), int(j)) for j in order[a0[i]:])
    return out
