"""Pins of the CPU oracle against facts other than itself.

Each test ties an oracle function to a closed form, a textbook identity, a
worked example of the paper, or brute force on tiny inputs, so that a
dropped term, a wrong sign or a swapped index in the oracle fails here.
"""
import itertools
import json
import os
import random

import mpmath
import numpy as np
import pytest

from oracle import factor, canonical
from oracle.atoms import atoms
from oracle.ddf import certify_irreducible, ddf_degrees
from oracle.recombine import (accept, band_pairs, expand, expand_values,
                              recombine_a, value)
from oracle.reduction import reduce_poly
from oracle.roots import complex_roots
from oracle.sturm import real_root_count
from oracle.zpoly import (is_squarefree, pdivmod_monic, peval, pmul, psub,
                          padd, primitive, trim)
from workloads import poly_mul, random_monic


def prod(polys):
    acc = [1]
    for f in polys:
        acc = pmul(acc, f)
    return acc


# ---------------------------------------------------------------- Z[x] basics
def test_divmod_identity():
    rng = random.Random(7)
    for _ in range(200):
        a = [rng.randint(-50, 50) for _ in range(rng.randint(1, 12))]
        b = [rng.randint(-9, 9) for _ in range(rng.randint(0, 6))] + [1]
        q, r = pdivmod_monic(a, b)
        assert padd(pmul(q, b), r) == trim(a)
        assert len(trim(r)) < len(b) or trim(r) == [0]


def test_squarefree():
    assert is_squarefree([1, 0, -10, 0, 1])
    assert not is_squarefree(pmul([-1, 1], pmul([-1, 1], [2, 1])))
    assert not is_squarefree(pmul([1, 0, 1], [1, 0, 1]))


# ---------------------------------------------------------------- Sturm count
def test_sturm_closed_forms():
    assert real_root_count(prod([[-i, 1] for i in range(1, 11)])) == 10
    assert real_root_count([1, 0, -10, 0, 1]) == 4          # Eq. 6: four real roots
    assert real_root_count([1, 0, 1]) == 0
    for m in (5, 6, 12, 30):                                 # x^m - 1: roots +-1 only
        assert real_root_count([-1] + [0] * (m - 1) + [1]) == (2 if m % 2 == 0 else 1)
    # Chebyshev T_n (non-monic, integer) has n real roots
    t0, t1 = [1], [0, 1]
    for n in range(2, 12):
        t0, t1 = t1, psub(pmul([0, 2], t1), t0)
        assert real_root_count(t1) == n


def test_sturm_against_eigenvalues():
    rng = np.random.default_rng(11)
    for _ in range(30):
        p = random_monic(rng, int(rng.integers(3, 16)), -20, 20)
        if not is_squarefree(p):
            continue
        z = np.roots([float(c) for c in reversed(p)])
        # count only unambiguous cases
        im = np.sort(np.abs(z.imag))
        r = int(np.sum(im < 1e-7))
        if r < len(im) and im[r] < 1e-3:
            continue
        assert real_root_count(p) == r


# ---------------------------------------------------------------- roots
def test_roots_newton_identities():
    rng = np.random.default_rng(3)
    for d in (5, 17, 40):
        p = random_monic(rng, d, -100, 100)
        z = complex_roots(p)
        with mpmath.workdps(60):
            s1 = mpmath.fsum(z)
            s2 = mpmath.fsum(w * w for w in z)
            assert abs(s1 + p[-2]) < 1e-45
            assert abs(s2 - (p[-2] ** 2 - 2 * p[-3])) < 1e-40
            for w in z:
                assert abs(mpmath.polyval([mpmath.mpf(c) for c in reversed(p)], w)) < 1e-35 * (1 + abs(w)) ** d * 100 ** 1


def test_rho_definition_sqrt2():
    # roots of x^2 - 2 are +-sqrt2; rho = (frac(-sqrt2), frac(sqrt2))
    _, r, els = reduce_poly([-2, 0, 1])
    assert r == 2 and [e.kind for e in els] == ["real", "real"]
    with mpmath.workdps(60):
        s2 = mpmath.sqrt(2)
        assert abs(els[0].rho - (2 - s2)) < 1e-50
        assert abs(els[1].rho - (s2 - 1)) < 1e-50


def test_pair_trace_parts():
    # x^2 + x + 1: one conjugate pair, z + conj z = -1, z^2 + conj z^2 = -1
    _, r, els = reduce_poly([1, 1, 1])
    assert r == 0 and len(els) == 1 and els[0].kind == "pair"
    assert abs(els[0].t1 + 1) < 1e-50 and abs(els[0].t2 + 1) < 1e-50 and abs(els[0].rho) < 1e-50


# ---------------------------------------------------------------- value/accept, EXPAND, FIND's set
def test_value_accept_and_complement_symmetry():
    rng = random.Random(5)
    M = 1 << 20
    for _ in range(30):
        n = rng.randint(2, 9)
        w = [rng.randrange(M) for _ in range(n - 1)]
        w.append((-sum(w)) % M)                          # whole set sums to an integer
        full = (1 << n) - 1
        for s in range(1 << n):
            a = accept(value(s, w, M), M, 3)
            b = accept(value(full ^ s, w, M), M, 3)
            assert a == b                                 # Section 3.1 symmetry
        assert accept(value(0, w, M), M, 0) and accept(value(full, w, M), M, 0)


def test_expand_is_sorted_subset_sums():
    rng = random.Random(9)
    M = 1 << 16
    w = [rng.randrange(M) for _ in range(6)]
    vals = expand_values(w, M)
    brute = [sum(c for c, bit in zip(w, bits) if bit) % M
             for bits in itertools.product([0, 1], repeat=6)]
    # itertools order is big-endian in bits; compare as multisets, and per pattern
    assert sorted(vals) == sorted(brute) == expand(w, M)
    for s in range(64):
        assert vals[s] == sum(w[i] for i in range(6) if s >> i & 1) % M


def test_band_pairs_equals_scan_on_concatenation():
    # Meet in the middle finds exactly the patterns RECOMBINE_A finds.
    rng = random.Random(13)
    M = 1 << 24
    for _ in range(20):
        na, nb = rng.randint(1, 5), rng.randint(1, 5)
        w = [rng.randrange(M) for _ in range(na + nb)] + [rng.randrange(M)]   # last = fixed element
        W = rng.choice([0, 5, 1 << 14])
        scan = set(recombine_a(w, M, W))
        alpha = expand_values(w[:na], M)
        beta = expand_values(w[na:na + nb], M)
        mitm = {i | (j << na) for (i, j) in band_pairs(alpha, beta, M, W)}
        assert scan == mitm


def test_band_pairs_sorted_equals_brute_force():
    # The sorted-list meet in the middle gives the brute-force pair set for
    # M = 2^64, with windows that run over 2^64 -> 0, zero weights (many equal
    # values) and the empty window.
    from oracle.recombine import band_pairs_sorted
    rng = random.Random(17)
    M = 1 << 64
    for trial in range(30):
        na, nb = rng.randint(0, 6), rng.randint(0, 6)
        if trial % 5 == 0:
            wa = [rng.randrange(8) for _ in range(na)]
            wb = [(-rng.randrange(8)) % M for _ in range(nb)]
        else:
            wa = [rng.randrange(M) for _ in range(na)]
            wb = [rng.randrange(M) for _ in range(nb)]
        if na and nb and trial % 3 == 0:
            wb[0] = (M - wa[0] + rng.randrange(-3, 4)) % M          # a pair straddling 0
        W = rng.choice([0, 2, 1 << 40, 1 << 62])
        brute = band_pairs(expand_values(wa, M), expand_values(wb, M), M, W)
        assert band_pairs_sorted(wa, wb, W) == brute


def test_recombine_vectorised_equals_loop():
    rng = random.Random(21)
    M = 1 << 62
    w = [rng.randrange(M) for _ in range(19)]
    # plant an integral subset
    w[3] = (-(w[0] + w[5] + w[11])) % M
    fast = recombine_a(w, M, 1 << 30)
    slow = [s for s in range(1 << 18) if accept(value(s, w, M), M, 1 << 30)]
    assert fast == slow and any(s == (1 | 8 | 32 | 2048) for s in fast)


def test_atoms():
    # divisors {0,1}, {0,1,2} of a 5-element set -> atoms {0,1}, {2}, {3,4}
    at = atoms(5, [{0, 1}, {0, 1, 2}])
    assert sorted(map(sorted, at)) == [[0, 1], [2], [3, 4]]
    assert atoms(3, []) == [frozenset({0, 1, 2})]


# ---------------------------------------------------------------- whole factorisation
def brute_factor(p):
    """Root-free brute force: repeatedly divide out the smallest-degree monic
    integer divisor, searched over the box given by the Cauchy root bound."""
    p = trim(p)
    out = []
    while len(p) > 2:
        d = len(p) - 1
        R = 1 + max(abs(c) for c in p[:-1])
        found = None
        for e in range(1, d // 2 + 1):
            from math import comb
            ranges = []
            for k in range(e):
                bound = comb(e, k) * R ** (e - k)
                if k == 0 and p[0] != 0:
                    ranges.append([s * v for v in range(1, abs(p[0]) + 1) if p[0] % v == 0 for s in (1, -1)])
                else:
                    ranges.append(range(-bound, bound + 1))
            for q in itertools.product(*ranges):
                cand = list(q) + [1]
                _, r = pdivmod_monic(p, cand)
                if r == [0]:
                    found = cand
                    break
            if found:
                break
        if not found:
            break
        out.append(found)
        p, _ = pdivmod_monic(p, found)
    out.append(p)
    return canonical(out)


def test_brute_force_tiny_all():
    count = 0
    for d in (2, 3, 4):
        for coeffs in itertools.product(range(-2, 3), repeat=d):
            p = list(coeffs) + [1]
            if not is_squarefree(p):
                continue
            assert factor(p).factors == brute_factor(p), p
            count += 1
    assert count > 500


def test_brute_force_tiny_sampled():
    rng = random.Random(17)
    for _ in range(25):
        d = rng.choice([5, 6])
        p = [rng.randint(-3, 3) for _ in range(d)] + [1]
        if rng.random() < 0.5:                         # make some reducible
            e = rng.randint(1, d - 1)
            p = pmul([rng.randint(-3, 3) for _ in range(e)] + [1],
                     [rng.randint(-3, 3) for _ in range(d - e)] + [1])
        if not is_squarefree(p):
            continue
        assert factor(p).factors == brute_factor(p), p


def cyclotomic(k, cache={}):
    """Phi_k by the textbook recursion x^k - 1 = prod_{j | k} Phi_j."""
    if k not in cache:
        num = [-1] + [0] * (k - 1) + [1]
        for j in range(1, k):
            if k % j == 0:
                num, r = pdivmod_monic(num, cyclotomic(j))
                assert r == [0]
        cache[k] = num
    return cache[k]


def test_cyclotomic_closed_forms():
    assert cyclotomic(12) == [1, 0, -1, 0, 1]
    assert cyclotomic(30) == [1, 1, 0, -1, -1, -1, 0, 1, 1]
    assert min(cyclotomic(105)) == -2                  # the first cyclotomic with a coefficient -2
    for m in (12, 30):
        res = factor([-1] + [0] * (m - 1) + [1])
        assert res.method == "exhaustive"
        assert res.factors == canonical([cyclotomic(k) for k in range(1, m + 1) if m % k == 0])


@pytest.mark.slow
def test_phi105():
    # Phi_105 is reducible modulo every prime, so no degree sieve can certify
    # it; the scan (n = 24) proves it irreducible.
    assert not certify_irreducible(cyclotomic(105), max_primes=15)[0]
    res = factor(cyclotomic(105))
    assert res.factors == [cyclotomic(105)] and res.n == 24 and res.r == 0


def sqrt_shift_product(f, m):
    """f(x - sqrt m) * f(x + sqrt m) in Z[x], by arithmetic in Z[sqrt m][x]
    (pairs (a, b) meaning a + b sqrt m)."""
    def mul(P, Q):
        out = [(0, 0)] * (len(P) + len(Q) - 1)
        for i, (a, b) in enumerate(P):
            for j, (c, e) in enumerate(Q):
                x, y = out[i + j]
                out[i + j] = (x + a * c + m * b * e, y + a * e + b * c)
        return out
    def compose(sign):                                  # f(x + sign*sqrt m)
        acc = [(0, 0)]
        for c in reversed(f):
            acc = mul(acc, [(0, sign), (1, 0)])
            acc[0] = (acc[0][0] + c, acc[0][1])
        return acc
    prodp = mul(compose(-1), compose(1))
    assert all(b == 0 for _, b in prodp)
    return trim([a for a, _ in prodp])


def test_swinnerton_dyer():
    f1 = [-2, 0, 1]                                     # prod (x +- sqrt2)
    f2 = sqrt_shift_product(f1, 3)
    assert f2 == [1, 0, -10, 0, 1]                      # Eq. 6
    res = factor(f2)
    assert res.factors == [f2] and res.n == 4 and res.r == 4
    # Every real factor has a dual with b_{e-1} = 0 (Section 2): candidates
    # exist, none verifies.  The pair {sqrt2+sqrt3, -sqrt2-sqrt3} sums to 0;
    # its product is x^2 - 5 - 2 sqrt6 (Eq. 7 with its constant corrected).
    assert len(res.candidates) >= 1 and res.verified == []
    f3 = sqrt_shift_product(f2, 5)
    assert f3 == [576, 0, -960, 0, 352, 0, -40, 0, 1]
    res3 = factor(f3)
    assert res3.factors == [f3] and res3.r == 8 and len(res3.candidates) >= 7 and res3.verified == []


def test_linear_split():
    p = prod([[-i, 1] for i in range(1, 11)])
    res = factor(p)
    assert res.factors == [[-i, 1] for i in range(10, 0, -1)]
    assert len(res.candidates) == 2 ** 9 - 1            # every rho is 0: every pattern is a candidate


def test_known_products_and_invariant():
    rng = np.random.default_rng(23)
    for _ in range(6):
        fs = [random_monic(rng, int(rng.integers(2, 9)), -20, 20) for _ in range(int(rng.integers(2, 4)))]
        p = [1]
        for f in fs:
            p = poly_mul(p, f)
        if not is_squarefree(p):
            continue
        res = factor(p)
        assert prod(res.factors) == p
        # every construction factor is a product of returned factors
        for f in fs:
            sub = [g for g in res.factors if pdivmod_monic(f, g)[1] == [0]]
            assert sub
        # the certificate route agrees with the scan
        cert = factor(p, construction=fs, max_scan_n=0)
        assert cert.factors == res.factors


# ---------------------------------------------------------------- DDF certificates
def test_ddf_degrees_small():
    assert ddf_degrees([1, 0, 1], 3) == {2: 1}          # x^2+1 irreducible mod 3
    assert ddf_degrees([1, 0, 1], 5) == {1: 2}          # splits mod 5 (2^2 = -1)
    assert ddf_degrees([-1, -1, 0, 0, 0, 1], 7) is not None


def test_certificates():
    assert certify_irreducible([-1, -1, 0, 0, 0, 1])[0]           # x^5 - x - 1
    assert certify_irreducible(cyclotomic(7))[0]
    assert not certify_irreducible([1, 0, 0, 0, 1], max_primes=20)[0]   # x^4+1: reducible mod every prime
    assert not certify_irreducible(pmul([1, 0, 1], [2, 0, 1]), max_primes=20)[0]


# ---------------------------------------------------------------- splat sort and query (Algorithms D, E)
def test_splat_sorts_and_keeps_every_value():
    """SPLAT's compacted output is the sorted input (Section 3.4): random
    values, values crowded into a few home cells, and values at the top end
    that overflow past the last home cell."""
    from oracle.splat import compact, home_cell, splat
    rng = random.Random(3)
    for vals, k in ([rng.randrange(1 << 64) for _ in range(3000)], 4096), \
                   (rng.sample(range(1 << 20), 500), 1024), \
                   ([(1 << 64) - 1 - i for i in range(300)], 512):
        cells, visited = splat(vals, k, home_cell(k, 64))
        assert compact(cells) == sorted(vals)
        assert visited >= len(vals)
        for i, c in enumerate(cells):                # at or after its home cell, no gap in between
            if c is not None:
                h = (c * k) >> 64
                assert h <= i and all(x is not None for x in cells[h:i + 1])


def test_splat_layout_does_not_depend_on_insertion_order():
    """The final array is the same for any insertion order: what lets a
    concurrent build be compared with the sequential one cell by cell."""
    from oracle.splat import home_cell, splat
    rng = random.Random(4)
    vals = [rng.randrange(1 << 40) for _ in range(1500)]
    vals += [v + 1 for v in vals[:200]]               # neighbours: long runs of full cells
    vals = list(set(vals))
    ref, _ = splat(vals, 2048, home_cell(2048, 40))
    for _ in range(3):
        rng.shuffle(vals)
        assert splat(vals, 2048, home_cell(2048, 40))[0] == ref


@pytest.mark.parametrize("c,lo,hi", [(2, 2 * np.log(2), 2.0), (4, 4 * np.log(4 / 3), 4 / 3)])
def test_splat_constant_within_theorem_bounds(c, lo, hi):
    """Theorem 3.4.2: for k uniform values in c*k cells, INSERT looks at C*k
    cells with c log(c/(c-1)) < C < c/(c-1) (1.386 < C < 2 for c = 2)."""
    from oracle.splat import home_cell, splat
    rng = random.Random(5)
    k = 1 << 14
    vals = [rng.randrange(1 << 64) for _ in range(k)]
    _, visited = splat(vals, c * k, home_cell(c * k, 64))
    assert lo < visited / k < hi


def test_query_band_is_a_filter():
    from oracle.splat import home_cell, query_band, splat
    rng = random.Random(6)
    k = 1 << 11
    vals = list({rng.randrange(1 << 32) for _ in range(k)})
    home = home_cell(2 * k, 32)
    cells, _ = splat(vals, 2 * k, home)
    for _ in range(300):
        a = rng.randrange(1 << 32)
        b = min((1 << 32) - 1, a + rng.choice([0, 5, 1 << 16, 1 << 22]))
        got = query_band(cells, home, a, b)
        assert sorted(v for _, v in got) == sorted(v for v in vals if a <= v <= b)
        assert all(cells[i] == v for i, v in got)


def test_printed_query_misses_what_the_band_query_finds():
    """Reading of QUERY: starting at the target's home cell, the printed QUERY
    never looks at an accepted value whose home cell is the one before."""
    from oracle.splat import home_cell, query_band, query_printed, splat
    bits, k, W = 16, 8, 4
    y, x = (1 << bits) // 8 - 1, (1 << bits) // 8 + 1   # home cells 0 and 1, |x - y| = 2 <= W
    cells, _ = splat([y], k, home_cell(k, bits), tail=4)
    assert not query_printed(cells, k, bits, x, lambda d: abs(d) <= W)
    assert query_band(cells, home_cell(k, bits), x - W, x + W) == [(0, y)]


@pytest.mark.parametrize("n_a,n_b,shift", [(5, 6, 3), (7, 8, 8), (8, 8, 10)])
def test_splat_match_equals_brute_force(n_a, n_b, shift):
    """RECOMBINE_E with the band query finds exactly the pairs in the circular
    window, including windows that wrap past 0."""
    from oracle.splat import splat_match
    rng = random.Random(n_a + 17 * n_b)
    M = 1 << 64
    wa = [rng.randrange(M) for _ in range(n_a)]
    wb = [rng.randrange(M) for _ in range(n_b)]
    wb[1] = (-(wa[0] + wa[2])) % M
    W = M >> shift
    exp = band_pairs(expand_values(wa, M), expand_values(wb, M), M, W)
    assert (0, 0) in exp and (5, 2) in exp
    assert splat_match(wa, wb, W) == exp


# ---------------------------------------------------------------- any p in Z[x] (Section 2's reductions)
def _group_by_mult(parts):
    """Multiply the parts of equal multiplicity together: {m: product}."""
    out = {}
    for f, m in parts:
        out[m] = pmul(out.get(m, [1]), f)
    return out


def test_yun_textbook_example():
    from oracle.squarefree import yun
    pp = [1]
    for f, m in (([-1, 1], 1), ([2, 1], 2), ([1, 0, 1], 3)):
        for _ in range(m):
            pp = pmul(pp, f)
    assert yun(pp) == [([-1, 1], 1), ([2, 1], 2), ([1, 0, 1], 3)]


def test_yun_invariants_on_random_constructions():
    """prod a_i^i == pp, every a_i square-free, pairwise coprime, and equal
    to the product of the construction's pieces of multiplicity i."""
    from oracle.squarefree import expand, yun
    from oracle.zpoly import is_squarefree
    rng = random.Random(21)
    for _ in range(12):
        pieces = []
        while len(pieces) < 4:
            f = [rng.randint(-5, 5) for _ in range(rng.randint(1, 4))] + [rng.choice([1, 2, 3])]
            f = trim(f)
            if len(f) > 1 and f[0] != 0:
                pieces.append((f, rng.randint(1, 3)))
        pp = expand(1, pieces)
        if not all(is_squarefree(primitive(g)) for g, _ in pieces):
            continue
        res = yun(primitive(pp))
        assert expand(1, res) == primitive(pp)
        for a, _ in res:
            assert is_squarefree(a)
        for (a, _), (b, _) in itertools.combinations(res, 2):
            assert is_squarefree(pmul(a, b))                      # coprime square-free parts
        if len({tuple(primitive(g)) for g, _ in pieces}) == 4 and is_squarefree(expand(1, [(g, 1) for g, _ in pieces])):
            want = {m: primitive(f) for m, f in _group_by_mult(pieces).items()}
            assert {m: f for f, m in res} == want


def test_factor_general_constructions():
    """content * prod f^m with irreducible f of known factorisation: monic
    factors the oracle certified (degree 12, coefficients in [-10, 10]) and
    Eisenstein polynomials (2x + 1; 3x^2 - 2 at 2; 5x^3 + 3x + 3 at 3)."""
    from oracle.squarefree import expand, factor_general
    recs = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cfg1.json")))
    monic = [f for r in recs for f in r["factors"] if len(f) > 2][:2]
    eis = [[1, 2], [-2, 0, 3], [3, 3, 0, 5]]
    for c, fs in ((-6, [(eis[0], 2), (eis[1], 1), ([0, 1], 3)]),
                  (1, [(monic[0], 2), (eis[2], 1)]),
                  (5, [(eis[1], 3), ([-1, 1], 1), ([1, 1], 2)])):
        got_c, got = factor_general(expand(c, fs))
        assert got_c == c
        assert got == sorted(fs, key=lambda fm: (len(fm[0]) - 1, tuple(fm[0]), fm[1]))


def test_squarefree_host_call_equals_oracle():
    """rfr_squarefree (host code of the library, no GPU) against the oracle's
    Yun: the same content, and per multiplicity the same product of parts."""
    from paper_2410_15880_b300.build import build
    build()
    import paper_2410_15880_b300 as P
    from oracle.squarefree import content, expand, yun
    rng = random.Random(8)
    cases = [[1, 0, -10, 0, 1], [0, 0, 3, 6], [-4, 0, 9], [7], [1, 2, 1], [2, 3, 1]]
    for _ in range(20):
        pieces = [(trim([rng.randint(-4, 4) for _ in range(rng.randint(1, 3))] + [rng.choice([1, 2, 3, -2])]),
                   rng.randint(1, 3)) for _ in range(3)]
        pieces = [(f, m) for f, m in pieces if len(f) > 1]
        p = expand(rng.choice([1, -1, 3, -10]), pieces)
        if max(abs(x) for x in p) < 1 << 40 and len(p) > 1:
            cases.append(p)
    for p in cases:
        r = P.squarefree(p)
        assert r.ok, p
        c, pp = content(p)
        assert r.content == c
        assert _group_by_mult(r.factors) == _group_by_mult(yun(pp)), p
        assert expand(r.content, r.factors) == trim(p)


def test_squarefree_host_call_errors():
    from paper_2410_15880_b300.build import build
    build()
    import paper_2410_15880_b300 as P
    assert P.squarefree([0, 0, 0]).status == -1                   # the zero polynomial
    assert P.squarefree([5]).ok and P.squarefree([5]).content == 5
    big = [1] * 20 + [1000]                                        # no monic transform on this path
    r = P.squarefree(big)
    assert r.ok and r.content == 1 and r.factors == [(big, 1)]


# ---------------------------------------------------------------- Algorithm B (search-tree pruning)
def test_prune_jump_paper_example():
    """Section 3.2's example: rho = (0.1, 0.2, 0.4, 0.8, ...), s ends in 1000
    and has value 0.2; 0.2 + 0.1 + 0.2 + 0.4 = 0.9 < 1, so the next seven
    patterns are skipped (a jump of 2^3).  From value 0.5 only 2^2."""
    from oracle.prune import jump_exponent
    M, W = 1000, 5
    ws = [100, 200, 400, 800]
    sigma = [0, 100, 300, 700, 1500]
    assert jump_exponent(200, 3, ws, sigma, M, W) == 3
    assert jump_exponent(500, 3, ws, sigma, M, W) == 2
    assert jump_exponent(200, 1, ws, sigma, M, W) == 1              # at most the trailing zeros of s
    assert jump_exponent(2, 3, ws, sigma, M, W) == 3                # 2 + 100 > W: nothing near 0 either
    assert jump_exponent(960, 3, ws, sigma, M, W) == 0              # 960 + 100 reaches the band at 1


@pytest.mark.parametrize("m,shift", [(10, 3), (12, 6), (14, 10)])
def test_prune_equals_recombine_a(m, shift):
    """RECOMBINE_B accepts exactly the patterns RECOMBINE_A accepts."""
    from oracle.prune import dist, recombine_b
    rng = random.Random(m)
    M = 1 << 64
    w = [rng.randrange(M) for _ in range(m)]
    w[3] = (-(w[0] + w[5])) % M
    W = M >> shift
    got, visited, _ = recombine_b(w, M, W)
    exp = {s for s in range(1 << m) if dist(sum(w[i] for i in range(m) if (s >> i) & 1), M) <= W}
    assert set(got) == exp and len(got) == len(exp)
    assert (1 | (1 << 3) | (1 << 5)) in exp and 0 in exp
    assert visited < (1 << m)


def test_prune_theorem_3_2_1_ratio():
    """Theorem 3.2.1: patterns / visited is about 2^l / l, l = floor(sqrt(2m))
    (for uniform values; the theorem's estimate drops the largest jumps)."""
    from oracle.prune import improvement_ratio, recombine_b
    M, m = 1 << 64, 16
    ratios = []
    for seed in range(6):
        rng = random.Random(100 + seed)
        w = [rng.randrange(M) for _ in range(m)]
        ratios.append((1 << m) / recombine_b(w, M, M >> 40)[1])
    mean = sum(ratios) / len(ratios)
    assert 0.5 < mean / improvement_ratio(m) < 2.0
