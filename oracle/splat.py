"""Splat sort (Algorithm D, Section 3.4) and its query (Algorithm E,
Section 3.5 and Section 4), sequential and plain, to check the GPU's splat
match against.  Test infrastructure: only tests, the smoke check and the
bench's CPU baseline use this package.

The splat array has k home cells.  A value x in [0, 2^bits) (the paper's
x in [0, 1) times 2^bits) has home cell floor(k x / 2^bits).  INSERT looks
at cells from the home cell on: an empty cell takes the carried value; a
full one keeps the smaller of its value and the carried one and the larger
moves on to the next cell.

Readings (where the printed algorithms are garbled or fall short):
- INSERT's step to the next cell is linear, into an overflow tail past the
  k home cells, not circular: with the circular step, values carried past
  the last cell land in front of the smallest ones and the array is no
  longer sorted in index order.
- QUERY as printed stops at the first accepted value and at the first cell
  above its target, and starts at the target's home cell; it misses accepted
  values that sit below that cell or after the first hit.  query_band
  reports every value of a band instead; query_printed keeps the printed
  form, to show the difference.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple


def splat(items: Sequence[int], k: int, home: Callable[[int], int], tail: int = 1 << 12):
    """SPLAT of the given items (distinct integers, ordered as integers) into
    k home cells plus `tail` overflow cells; home(item) in [0, k) must be
    non-decreasing in the item.  Returns (cells, visited): cells is a list of
    k + tail entries (None = empty); visited counts the cells INSERT looked at
    over all items (Theorem 3.4.2's C times the number of items)."""
    cells: List[Optional[int]] = [None] * (k + tail)
    visited = 0
    for x in items:
        i = home(x)
        while True:                                   # INSERT
            visited += 1
            y = cells[i]
            if y is None:
                cells[i] = x
                break
            if y > x:                                 # the smaller value stays, the larger moves on
                cells[i], x = x, y
            i += 1
            if i == len(cells):
                raise OverflowError("splat: insertion ran past the overflow tail")
    return cells, visited


def compact(cells) -> List[int]:
    """Step 12 of SPLAT: the non-empty cells in index order."""
    return [c for c in cells if c is not None]


def home_cell(k: int, bits: int) -> Callable[[int], int]:
    """floor(k x) for x = value / 2^bits."""
    return lambda v: (v * k) >> bits


def query_band(cells, home: Callable[[int], int], lo: int, hi: int) -> List[Tuple[int, int]]:
    """Every (index, item) with lo <= item <= hi in a splat array.  The scan
    starts at home(lo): an item sits at or after its home cell, and the
    cells between its home cell and its place are all full.  It stops at the
    first item above hi, or at the first empty cell at or past home(hi)."""
    out = []
    i, h_hi = home(lo), home(hi)
    while i < len(cells):
        c = cells[i]
        if c is None:
            if i >= h_hi:
                break
        elif c > hi:
            break
        elif c >= lo:
            out.append((i, c))
        i += 1
    return out


def query_printed(cells, k: int, bits: int, x: int, accept: Callable[[int], bool]) -> bool:
    """QUERY as the paper prints it (Section 3.5): from x's home cell, true at
    the first accepted cell, false at an empty cell or a cell above x; the
    step is circular over the k home cells."""
    i = (x * k) >> bits
    for _ in range(k):
        c = cells[i]
        if c is None:
            return False
        if accept(x - c):
            return True
        if c > x:
            return False
        i = (i + 1) % k
    return False


def splat_match(w_a: Sequence[int], w_b: Sequence[int], window: int, tail: int = 1 << 12):
    """RECOMBINE_E with the band query, M = 2^64: beta = SPLAT of the half-b
    sums sum_{j in s_b} w_b[j] (mod 2^64) with c = 2 (2^(n_b+1) home cells),
    each item carrying its pattern (item = sum * 2^n_b + s_b); then for every
    pattern s_a of half a, the betas within the circular window of
    -alpha(s_a) (Eq. 9) are found with query_band (two bands where the window
    wraps past 0).  Returns the set of (s_a, s_b)."""
    M = 1 << 64
    n_b = len(w_b)
    k = 2 << n_b
    hb = 1 << n_b

    def sums(w):
        v = [0]
        for x in w:
            v = v + [(s + x) % M for s in v]
        return v

    alpha, beta = sums(w_a), sums(w_b)
    home = lambda item: ((item >> n_b) * k) >> 64  # noqa: E731
    cells, _ = splat([beta[s] * hb + s for s in range(len(beta))], k, home, tail)
    out = set()
    for s_a, a in enumerate(alpha):
        t = (-a) % M
        lo, hi = t - window, t + window
        bands = [(lo, hi)] if lo >= 0 and hi < M else [(lo % M, M - 1), (0, hi % M)]
        for l, h in bands:
            for _, item in query_band(cells, home, l * hb, h * hb + hb - 1):
                out.add((s_a, item & (hb - 1)))
    return out
