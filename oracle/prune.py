"""Algorithm B (Section 3.2, RECOMBINE_B): search-tree pruning over the
2^m patterns of m elements, sequential and plain, to check the GPU's pruned
search against.  Test infrastructure: only tests, the smoke check and the
bench's CPU baseline use this package.

Values are fixed point: an element is w = round(rho * M) with M = 2^64 (or
any M), a pattern's value is the sum of its elements' w modulo M.  The
elements are sorted ascending; sigma_i is the sum of the i smallest.

Readings:
- Acceptance is circular (Eq. 9): dist(v) = min(v mod M, M - v mod M) <= W.
- The jump.  After visiting s with value x, the next 2^j - 1 patterns
  (j at most the number of trailing zero bits of s) have values x + t for the
  non-empty sums t of the j smallest elements, so they lie in
  [x + w_1, x + sigma_j] as integers.  None of them is accepted when
  x + w_1 > W and x + sigma_j < M - W: the paper's condition
  value + sigma_j < 1, with the band around 0 as well as the one around 1.
  j is the largest such exponent.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def dist(v: int, M: int) -> int:
    v %= M
    return min(v, M - v)


def jump_exponent(x: int, c: int, w_sorted: Sequence[int], sigma: Sequence[int], M: int, W: int) -> int:
    """The largest j <= c such that no pattern strictly between s and
    s + 2^j is accepted, for a pattern s with value x (0 <= x < M) and c
    trailing zero bits; w_sorted ascending, sigma[i] = sum of the i smallest
    (as integers, not reduced)."""
    if not w_sorted or x + w_sorted[0] <= W:
        return 0
    j = 0
    while j < c and j + 1 < len(sigma) and x + sigma[j + 1] < M - W:
        j += 1
    return j


def recombine_b(w: Sequence[int], M: int, W: int) -> Tuple[List[int], int, List[int]]:
    """RECOMBINE_B over all 2^m patterns of the m elements w (the caller
    leaves the fixed element out).  Returns (accepted patterns over the
    ORIGINAL element order, in visiting order, including 0; number of
    patterns visited; the sorting permutation)."""
    m = len(w)
    order = sorted(range(m), key=lambda i: w[i])
    ws = [w[i] % M for i in order]
    sigma = [0]
    for v in ws:
        sigma.append(sigma[-1] + v)
    out, visited = [], 0
    s = 0
    while s < (1 << m):
        visited += 1
        x = sum(ws[i] for i in range(m) if (s >> i) & 1) % M
        if dist(x, M) <= W:
            out.append(sum(1 << order[i] for i in range(m) if (s >> i) & 1))
        c = (s & -s).bit_length() - 1 if s else m
        j = jump_exponent(x, c, ws, sigma, M, W)
        s += 1 << j
    return out, visited, order


def improvement_ratio(m: int) -> float:
    """Theorem 3.2.1's expected ratio 2^l / l, l = floor(sqrt(2 m))."""
    l = int((2 * m) ** 0.5)
    return 2 ** l / l
