"""The splat match (Section 4, Algorithm E) on the GPU against the oracle:
the splat array cell by cell against the sequential SPLAT, Theorem 3.4.2's
constant, and the candidate sets against the brute-force and sorted pair
sets."""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import golden, to_u64, u64_tensor  # noqa: E402
from oracle.recombine import band_pairs, band_pairs_sorted, expand_values, expand_values_u64  # noqa: E402
from oracle.splat import compact, splat  # noqa: E402

M64 = 1 << 64
EMPTY = M64 - 1


@pytest.fixture(scope="module")
def P():
    import paper_2410_15880_b300 as P
    return P


def cell_values(w, n):
    """The stage's cell values e(s) = ((S(s) >> 1) & ~(2^n - 1)) | s, by definition."""
    S = expand_values_u64(w[:n]) if n else np.zeros(1, dtype=np.uint64)
    lm = np.uint64((1 << n) - 1)
    return ((S >> np.uint64(1)) & ~lm) | np.arange(1 << n, dtype=np.uint64)


@pytest.mark.parametrize("n", [0, 1, 5, 11, 12, 14])
def test_splat_array_equals_sequential_splat(P, n):
    rng = random.Random(40 + n)
    w = [rng.randrange(M64) for _ in range(max(n, 1))]
    gamma, ctr = P.stage_splat(u64_tensor(w), n)
    torch.cuda.synchronize()
    cells = to_u64(gamma)[:(2 << n) + 4096]
    e = [int(x) for x in cell_values(w, n)]
    ref, visited = splat(e, 2 << n, lambda v: v >> (62 - n), tail=4096)
    got = [None if int(c) == EMPTY else int(c) for c in cells]
    assert got == ref
    assert compact(got) == sorted(e)
    c = [int(x) for x in to_u64(ctr)]
    assert c[4] == 0 and c[5] >= len(e) and c[6] >= c[5]


def test_splat_constant(P):
    """Cells looked at per insertion (Theorem 3.4.2, c = 2: 1.386 < C < 2 for
    sequential insertion of uniform values).  Concurrent insertion looks at
    about as many cells."""
    rng = random.Random(9)
    n = 20
    w = [rng.randrange(M64) for _ in range(n)]
    _, ctr = P.stage_splat(u64_tensor(w), n)
    c = [int(x) for x in to_u64(ctr)]
    C = c[5] / (1 << n)
    print(f"splat n_b={n}: C = {C:.3f}, exchanges per insertion {c[6] / (1 << n):.3f}")
    assert c[4] == 0 and 1.3 < C < 2.1


def _splat_pairs(P, wa, w2a, wb, w2b, W, W2, cap=1 << 16):
    cand, ctr, _ = P.stage_splat_match(u64_tensor(wa or [0]) [:len(wa)], u64_tensor(w2a or [0])[:len(wa)],
                                       u64_tensor(wb or [0])[:len(wb)], u64_tensor(w2b or [0])[:len(wb)],
                                       W, W2, cap)
    torch.cuda.synchronize()
    c = [int(x) for x in to_u64(ctr)]
    na = len(wa)
    got = {(int(x) & ((1 << na) - 1), int(x) >> na) for x in to_u64(cand)[:min(c[2], cap)]}
    return got, c


@pytest.mark.parametrize("na,nb,shift", [(0, 1, 2), (3, 4, 3), (7, 8, 6), (10, 11, 10), (12, 13, 13)])
def test_splat_match_bruteforce(P, na, nb, shift):
    rng = random.Random(na * 7 + nb)
    wa = [rng.randrange(M64) for _ in range(na)]
    wb = [rng.randrange(M64) for _ in range(nb)]
    if na >= 2:
        wb[0] = (-(wa[0] + wa[1])) % M64
    W = M64 >> shift
    exp = band_pairs(expand_values(wa, M64), expand_values(wb, M64), M64, W)
    got, c = _splat_pairs(P, wa, [0] * na, wb, [0] * nb, W, 0)
    assert c[4] == 0 and c[3] == 1 and c[1] == len(exp)
    assert got == exp - {(0, 0)} and c[2] == len(got)


def test_splat_match_tr2(P):
    rng = random.Random(77)
    wa, wb = [rng.randrange(M64) for _ in range(8)], [rng.randrange(M64) for _ in range(9)]
    w2a, w2b = [rng.randrange(M64) for _ in range(8)], [rng.randrange(M64) for _ in range(9)]
    W, W2 = M64 >> 6, M64 >> 2
    pairs = band_pairs(expand_values(wa, M64), expand_values(wb, M64), M64, W) - {(0, 0)}
    t2a, t2b = expand_values(w2a, M64), expand_values(w2b, M64)
    exp = {(i, j) for i, j in pairs if min((t2a[i] + t2b[j]) % M64, (-(t2a[i] + t2b[j])) % M64) <= W2}
    got, c = _splat_pairs(P, wa, w2a, wb, w2b, W, W2)
    assert 0 < len(exp) < len(pairs) and got == exp and c[1] == len(pairs) + 1


@pytest.mark.parametrize("na,nb,shift", [(14, 15, 22), (20, 21, 34), (22, 23, 40)])
def test_splat_match_against_sorted_mitm(P, na, nb, shift):
    rng = random.Random(na + nb)
    wa = [rng.randrange(M64) for _ in range(na)]
    wb = [rng.randrange(M64) for _ in range(nb)]
    wb[3] = (-(wa[1] + wa[5] + wb[7])) % M64
    W = M64 >> shift
    exp = band_pairs_sorted(wa, wb, W)
    got, c = _splat_pairs(P, wa, [0] * na, wb, [0] * nb, W, 0, cap=1 << 20)
    assert (0b100010, (1 << 3) | (1 << 7)) in exp
    assert c[4] == 0 and got == exp - {(0, 0)} and c[1] == len(exp)


def test_splat_overflow_is_flagged(P):
    """Fourteen zero weights put 2^14 values in one home cell: an insertion
    runs past its step limit and the counters say so."""
    rng = random.Random(3)
    wb = [0] * 14 + [rng.randrange(M64) for _ in range(2)]
    _, ctr = P.stage_splat(u64_tensor(wb), 16)
    assert int(to_u64(ctr)[4]) == 1


def test_factor_splat_path_equals_goldens(P):
    """rfr_config.match_path = RFR_MATCH_SPLAT: every problem with 13 < n_b
    <= 30 through the splat match (clustered weights fall back to the table
    match); the factorisations equal the oracle's goldens and the default path's."""
    recs = golden("cfg3")[:6] + golden("cfg2")[:8] + golden("special")
    polys = [r["coeffs"] for r in recs]
    with P.Context(device=0) as auto, P.Context(device=0, match_path=P.RFR_MATCH_SPLAT) as sp:
        ra = auto.factor_batch(polys)
        rs = sp.factor_batch(polys)
    for r, a, s in zip(recs, ra, rs):
        assert a.ok and s.ok, r.get("name")
        assert a.factors == s.factors == r["factors"]
        assert a.diag["cand_post"] == s.diag["cand_post"]


@pytest.mark.parametrize("m", [60, 105])
def test_x_m_minus_1_every_match_path(P, m):
    """x^m - 1 = prod_{k | m} Phi_k (closed form, each Phi_k irreducible).  Its
    weights are sums of cosines with many exact coincidences: keys cluster
    (the fused and splat matches fall back to the table match) and many
    patterns that are not divisors have coefficients near integers."""
    from oracle import canonical
    from test_oracle_pins import cyclotomic
    p = [-1] + [0] * (m - 1) + [1]
    exp = canonical([cyclotomic(k) for k in range(1, m + 1) if m % k == 0])
    for mp in (P.RFR_MATCH_AUTO, P.RFR_MATCH_TABLES, P.RFR_MATCH_SPLAT):
        with P.Context(device=0, match_path=mp, max_candidates=1 << 21) as c:
            r = c.factor(p)
        assert r.ok, (mp, r.status)
        assert r.factors == exp
