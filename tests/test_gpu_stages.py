"""Stage-level parity of the CUDA path against the CPU oracle (through the C ABI).

K-a roots, K-b weights, K-c enumerate, K-c/K-d/K-e match and K-f verify, each
on seeded inputs, element by element where the result is unique."""
import functools
import random

import mpmath
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import coeff_tensor, golden, plans_numpy, to_u64, u64_tensor  # noqa: E402

M64 = 1 << 64


@pytest.fixture(scope="module")
def P():
    import paper_2410_15880_b300 as P
    P.lib()
    return P


def circ(y):
    y %= M64
    return min(y, M64 - y)


def small_set():
    recs = golden("cfg1") + golden("special") + golden("cfg2")[:6] + golden("cfg4_sample")[:12]
    return [r for r in recs if len(r["coeffs"]) > 2]


# ---------------------------------------------------------------- K-a
@pytest.mark.parametrize("mode", [0, 1])
def test_roots_within_radius_and_residual(P, mode):
    from oracle.roots import complex_roots
    recs = small_set()
    c, d = coeff_tensor([r["coeffs"] for r in recs])
    roots, radius, status = P.stage_roots(c, d, mode)
    torch.cuda.synchronize()
    R, rad, st = roots.cpu().numpy(), radius.cpu().numpy(), status.cpu().numpy()
    for i, r in enumerate(recs):
      assert st[i] == 0, r["name"]
      deg = len(r["coeffs"]) - 1
      ref = complex_roots(r["coeffs"])
      p = r["coeffs"]
      with mpmath.workdps(60):
        for j in range(deg):
            z = mpmath.mpc(mpmath.mpf(R[i, j, 0]) + mpmath.mpf(R[i, j, 1]),
                           mpmath.mpf(R[i, j, 2]) + mpmath.mpf(R[i, j, 3]))
            err = min(abs(z - w) for w in ref)
            assert err <= rad[i, j], (r["name"], j, float(err), rad[i, j])      # inclusion radius holds
            zh = mpmath.mpc(float(R[i, j, 0]), float(R[i, j, 2]))              # the FP64 part alone
            num = abs(mpmath.polyval([mpmath.mpf(x) for x in reversed(p)], zh))
            den = sum(abs(x) * abs(zh) ** k for k, x in enumerate(p))
            assert num / den <= 1e-10                                           # relative residual (FP64 bar)


# ---------------------------------------------------------------- K-b
def test_weights_against_oracle_rho(P):
    from oracle.reduction import elements_from_roots
    from oracle.roots import complex_roots
    from oracle.sturm import real_root_count
    recs = small_set()
    c, d = coeff_tensor([r["coeffs"] for r in recs])
    roots, radius, status = P.stage_roots(c, d)
    plans = plans_numpy(P.stage_weights(c, d, roots, radius, status))
    for i, r in enumerate(recs):
        pl = plans[i]
        assert pl["status"] == 0, r["name"]
        els = elements_from_roots(complex_roots(r["coeffs"]), real_root_count(r["coeffs"]))
        n = len(els)
        assert (pl["n"], pl["r"]) == (n, r["r"]), r["name"]
        assert pl["n_a"] == (n - 1) // 2 and pl["n_b"] == n - 1 - (n - 1) // 2
        W = int(pl["window"])
        with mpmath.workdps(60):
            for k, e in enumerate(els):
                assert pl["kind"][k] == e.degree
                ref = int(mpmath.nint(e.rho * M64)) % M64
                assert circ(int(pl["w"][k]) - ref) <= W, (r["name"], k)
                ref2 = int(mpmath.nint((e.t2 - mpmath.floor(e.t2)) * M64)) % M64
                assert circ(int(pl["w2"][k]) - ref2) <= int(pl["window2"]), (r["name"], k)
        # Vieta: all elements together sum to an integer
        assert circ(sum(int(x) for x in pl["w"][:n])) <= W


# ---------------------------------------------------------------- K-c plain
@pytest.mark.parametrize("h", [0, 1, 3, 5, 6, 7, 11, 14])
def test_enumerate_bit_exact(P, h):
    from oracle.recombine import expand_values
    from workloads import random_weights
    w = [int(x) for x in random_weights(100 + h, max(h, 1))][:h]
    keys = P.stage_enumerate(u64_tensor(w if h else [0]), h)
    got = [int(x) for x in to_u64(keys)]
    assert got == expand_values(w, M64)


def test_enumerate_large_properties(P):
    from oracle.recombine import value
    from workloads import random_weights
    h = 24
    w = [int(x) for x in random_weights(7, h)]
    keys = to_u64(P.stage_enumerate(u64_tensor(w), h))
    # sum over all s of key(s) = 2^(h-1) * sum(w)  (mod 2^64)
    assert int(keys.sum(dtype=np.uint64)) == (2 ** (h - 1) * sum(w)) % M64
    rng = random.Random(3)
    for s in [0, 1, (1 << h) - 1] + [rng.randrange(1 << h) for _ in range(200)]:
        assert int(keys[s]) == value(s, w, M64)


# ---------------------------------------------------------------- K-d sorted low lists (fused match)
@pytest.mark.parametrize("l,negate", [(0, False), (1, False), (5, True), (12, False), (13, True), (16, False),
                                      (20, True), (24, False)])
def test_lowlist_sorted_and_complete(P, l, negate):
    """The list is non-decreasing, its masks are every subset once, and each
    entry is the exact sum (mod 2^64) of the weights its mask names: the
    sorted EXPAND of Section 3.3 by its definition."""
    rng = random.Random(100 + l)
    w = [rng.randrange(M64) for _ in range(max(l, 1))]
    out, masks, _ = P.stage_lowlist(u64_tensor(w), l, negate)
    torch.cuda.synchronize()
    got = to_u64(out)
    m = masks.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.all(got[1:] >= got[:-1])                        # sorted
    assert np.array_equal(np.sort(m), np.arange(1 << l))      # every subset once
    s_ = np.zeros(1, dtype=np.uint64)                          # S(s) for s in pattern order, modulo 2^64
    for x in w[:l]:
        s_ = np.concatenate([s_, s_ + np.uint64((-x if negate else x) % M64)])
    assert np.array_equal(got, s_[m])


# ---------------------------------------------------------------- K-c/K-d/K-e match
def _expected_pairs(wa, w2a, wb, w2b, W, W2):
    from oracle.recombine import accept, band_pairs, expand_values
    alpha, beta = expand_values(wa, M64), expand_values(wb, M64)
    a2, b2 = expand_values(w2a, M64), expand_values(w2b, M64)
    pairs = band_pairs(alpha, beta, M64, W)
    return {(i, j) for (i, j) in pairs if accept((a2[i] + b2[j]) % M64, M64, W2)}


def _run_match(P, wa, w2a, wb, w2b, W, W2, cap=1 << 16, exact=False, fused=False):
    cand, ctr, _ = P.stage_match(u64_tensor(wa) if wa else u64_tensor([0])[:0],
                                 u64_tensor(w2a) if wa else u64_tensor([0])[:0],
                                 u64_tensor(wb) if wb else u64_tensor([0])[:0],
                                 u64_tensor(w2b) if wb else u64_tensor([0])[:0], W, W2, cap, exact=exact,
                                 fused=fused)
    torch.cuda.synchronize()
    ctr = [int(x) for x in ctr.cpu().numpy().view(np.uint64)]
    cnt = ctr[2]
    got = [int(x) for x in to_u64(cand)[:min(cnt, cap)]]
    na = len(wa)
    return {(s & ((1 << na) - 1), s >> na) for s in got}, ctr, got


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("seed,na,nb", [(1, 0, 0), (2, 0, 1), (3, 1, 1), (4, 2, 3), (5, 4, 4),
                                        (6, 5, 6), (7, 7, 8), (8, 9, 9), (9, 10, 11)])
def test_match_bruteforce(P, seed, na, nb, fused):
    if fused and na < 2:
        pytest.skip("the fused match needs two elements per half")
    rng = random.Random(seed)
    W = rng.choice([0, 3, 1 << 20, 1 << 52])
    wa = [rng.randrange(M64) for _ in range(na)]
    wb = [rng.randrange(M64) for _ in range(nb)]
    if na and nb:                                   # plant an integral subset across the halves
        wb[0] = (-(wa[0] + (wa[-1] if na > 1 else 0))) % M64
    w2a = [rng.randrange(M64) for _ in range(na)]
    w2b = [rng.randrange(M64) for _ in range(nb)]
    W2 = 1 << 63                                    # Tr_2 filter off
    got, ctr, raw = _run_match(P, wa, w2a, wb, w2b, W, W2, fused=fused)
    exp = _expected_pairs(wa, w2a, wb, w2b, W, W2)
    assert ctr[3] == 1                              # the empty pattern always matches
    assert got == exp - {(0, 0)}
    assert len(raw) == len(set(raw))                # every pair once
    assert ctr[4] == 0


def test_match_tr2_filter(P):
    rng = random.Random(42)
    na, nb = 8, 9
    wa = [rng.randrange(M64) for _ in range(na)]
    wb = [rng.randrange(M64) for _ in range(nb)]
    W = 1 << 58                                    # wide Tr_1 window: many pairs
    w2a = [rng.randrange(M64) for _ in range(na)]
    w2b = [rng.randrange(M64) for _ in range(nb)]
    W2 = 1 << 61
    got, ctr, _ = _run_match(P, wa, w2a, wb, w2b, W, W2)
    exp = _expected_pairs(wa, w2a, wb, w2b, W, W2)
    assert got == exp - {(0, 0)} and len(got) > 0
    assert ctr[2] == len(got) and ctr[1] >= ctr[2]


def test_match_degenerate_all_zero(P):
    # every weight 0 (e.g. all roots integers): every pattern is a candidate
    na, nb = 4, 5
    got, ctr, _ = _run_match(P, [0] * na, [0] * na, [0] * nb, [0] * nb, 5, 5)
    assert got == {(i, j) for i in range(1 << na) for j in range(1 << nb)} - {(0, 0)}


def test_match_candidate_cap(P):
    na, nb = 4, 5
    got, ctr, raw = _run_match(P, [0] * na, [0] * na, [0] * nb, [0] * nb, 5, 5, cap=10)
    assert ctr[2] == (1 << 9) - 1 and len(raw) == 10


@functools.lru_cache(maxsize=4)
def _scan(w, W):
    """RECOMBINE_A's accepted patterns (the oracle), shared by the layouts."""
    from oracle.recombine import recombine_a
    return frozenset(recombine_a(list(w), M64, W))


@pytest.mark.parametrize("layout", ["slack", "exact", "fused"])
@pytest.mark.parametrize("seed,na,nb", [(11, 14, 15), (12, 16, 16), (13, 17, 18)])
def test_match_several_tiles_against_scan(P, seed, na, nb, layout):
    """Sizes that span many buckets and CTAs, vs RECOMBINE_A on the concatenation,
    with the slack-region layout, the exact (count pass) layout and the fused
    match (many key units, several runs per half)."""
    exact, fused = layout == "exact", layout == "fused"
    rng = random.Random(seed)
    wa = [rng.randrange(M64) for _ in range(na)]
    wb = [rng.randrange(M64) for _ in range(nb)]
    # plant three integral subsets
    wb[2] = (-(wa[0] + wa[5] + wb[7])) % M64
    wa[9] = (-(wb[1] + wb[3])) % M64
    W = 1 << 30
    got, ctr, _ = _run_match(P, wa, [0] * na, wb, [0] * nb, W, 0, exact=exact, fused=fused)
    assert ctr[4] == 0
    scan = _scan(tuple(wa + wb + [0]), W) - {0}
    exp = {(s & ((1 << na) - 1), s >> na) for s in scan}
    assert got == exp and len(exp) >= 2


# ---------------------------------------------------------------- K-f verify
def test_verify_true_and_false_patterns(P):
    recs = [r for r in golden("cfg1") + golden("special") if len(r["factors"]) > 1 or r["name"].startswith("swinnerton")]
    c, d = coeff_tensor([r["coeffs"] for r in recs])
    roots, radius, status = P.stage_roots(c, d)
    plans_t = P.stage_weights(c, d, roots, radius, status)
    plans = plans_numpy(plans_t)
    R = roots.cpu().numpy()
    prob, lo, hi, expect_coeffs = [], [], [], []
    for i, r in enumerate(recs):
        pl = plans[i]
        n = int(pl["n"])
        for f in r["factors"]:
            # elements whose root is a root of f
            pat = 0
            for k in range(n):
                z = complex(R[i, pl["root0"][k], 0], R[i, pl["root0"][k], 2])
                val = abs(np.polyval(list(reversed(f)), z))
                scale = sum(abs(x) * abs(z) ** j for j, x in enumerate(f))
                if val <= 1e-8 * scale:
                    pat |= 1 << k
            prob.append(i); lo.append(pat); hi.append(0); expect_coeffs.append(f)
        if r["name"] == "swinnerton_dyer_f2":
            # the pair {sqrt2+sqrt3, -sqrt2-sqrt3}: Tr_1 = 0 but not a factor (Section 2)
            prob.append(i); lo.append(0b1001); hi.append(0); expect_coeffs.append(None)
    pt = torch.tensor(prob, dtype=torch.int32, device="cuda")
    res, co = P.stage_verify(c, d, roots, plans_t, pt, u64_tensor(lo), u64_tensor(hi), want_coeffs=True)
    res = res.cpu().numpy()
    co = co.cpu().numpy()
    for j, f in enumerate(expect_coeffs):
        if f is None:
            assert res[j] == 0
        else:
            assert res[j] == 1, (j, f)
            assert list(co[j, :len(f)]) == f


def test_match_clustered_keys_fit_one_unit(P):
    """Weights below 2^40 put all 2^14 keys of half a in one key unit, which
    the fused match's table still holds: its answer is the scan's, with no
    overflow."""
    from oracle.recombine import recombine_a
    rng = random.Random(77)
    na, nb = 14, 15
    wa = [rng.randrange(1 << 40) for _ in range(na)]
    wb = [rng.randrange(1 << 40) for _ in range(nb)]
    wa[0] = 0                                           # {a0} sums to an integer
    W = 1 << 20
    got, ctr, _ = _run_match(P, wa, [0] * na, wb, [0] * nb, W, 0, fused=True)
    assert ctr[4] == 0
    scan = set(recombine_a(wa + wb + [0], M64, W)) - {0}
    assert got == {(s & ((1 << na) - 1), s >> na) for s in scan} and (1, 0) in got


def test_match_clustered_keys_overflow_then_exact(P):
    """Weights below 2^40 put every key in one bucket: the fused match (the
    automatic choice) must report the overflow of its table, and the exact
    layout must give the scan's answer."""
    from oracle.recombine import recombine_a
    rng = random.Random(77)
    na, nb = 15, 15
    wa = [rng.randrange(1 << 40) for _ in range(na)]
    wb = [rng.randrange(1 << 40) for _ in range(nb)]
    wa[0] = 0                                           # {a0} sums to an integer
    W = 1 << 20
    _, ctr, _ = _run_match(P, wa, [0] * na, wb, [0] * nb, W, 0)
    assert ctr[4] == 1
    got, ctr2, _ = _run_match(P, wa, [0] * na, wb, [0] * nb, W, 0, exact=True)
    assert ctr2[4] == 0
    scan = set(recombine_a(wa + wb + [0], M64, W)) - {0}
    assert got == {(s & ((1 << na) - 1), s >> na) for s in scan} and (1, 0) in got


# ---------------------------------------------------------------- fused match at large sizes
@pytest.mark.parametrize("seed,na,nb,logW,tr2", [(31, 20, 21, 30, False), (32, 22, 22, 38, True),
                                               (33, 23, 24, 30, False)])
def test_match_fused_large_against_sorted_mitm(P, seed, na, nb, logW, tr2):
    """The fused match (sorted lists built by merging, key units in shared
    memory) at sizes with 2^7 runs per half and up to 2^10 key units, vs the
    sorted-list meet in the middle of the oracle.  Planted weights put pairs
    across the circular wrap in both directions and across the unit boundary
    at 2^63; three integral subsets are planted too."""
    from oracle.recombine import accept, band_pairs_sorted, expand_values_u64
    rng = random.Random(seed)
    wa = [rng.randrange(M64) for _ in range(na)]
    wb = [rng.randrange(M64) for _ in range(nb)]
    wa[0], wb[0] = M64 - 3, M64 - 2                   # K_a = 2^64 - 3 meets K_b = 2 (over the wrap)
    wa[1], wb[1] = 3, 2                               # K_a = 3 meets K_b = 2^64 - 2
    wa[2], wb[2] = (1 << 63) - 1, (1 << 63) - 1       # K_a just below 2^63, K_b just above
    wb[5] = (-(wa[4] + wa[7] + wb[9])) % M64
    wa[11] = (-(wb[12] + wb[13])) % M64
    W = 1 << logW
    if tr2:
        w2a = [rng.randrange(M64) for _ in range(na)]
        w2b = [rng.randrange(M64) for _ in range(nb)]
        W2 = 1 << 62
    else:
        w2a, w2b, W2 = [0] * na, [0] * nb, 0
    got, ctr, raw = _run_match(P, wa, w2a, wb, w2b, W, W2, cap=1 << 20, fused=True)
    pairs = band_pairs_sorted(wa, wb, W)
    if tr2:
        a2, b2 = expand_values_u64(w2a), expand_values_u64(w2b)
        pairs = {(i, j) for (i, j) in pairs if accept((int(a2[i]) + int(b2[j])) % M64, M64, W2)}
    assert ctr[4] == 0 and ctr[3] == 1
    assert got == pairs - {(0, 0)}
    assert len(raw) == len(set(raw)) and ctr[2] == len(raw)
    assert ctr[1] >= ctr[2] and ctr[0] >= ctr[1]
    if not tr2:                                       # planted pairs (Tr_2 may reject them otherwise)
        for pl in [(1, 1), (2, 2), (4, 4), (1 | 2, 1 | 2)]:
            assert pl in got


# ---------------------------------------------------------------- completeness at production sizes
_PROD_CACHE = {}


def _production_case(seed, na, nb, logW, tr2):
    """Weights (with planted integral subsets and pairs across the circular
    wrap) and the oracle's pair set (sorted meet in the middle, then the Tr_2
    test) for halves of na and nb elements; cached per argument tuple."""
    key = (seed, na, nb, logW, tr2)
    if key in _PROD_CACHE:
        return _PROD_CACHE[key]
    from oracle.recombine import accept, band_pairs_sorted, expand_values_u64
    rng = random.Random(seed)
    wa = [rng.randrange(M64) for _ in range(na)]
    wb = [rng.randrange(M64) for _ in range(nb)]
    wa[0], wb[0] = M64 - 3, M64 - 2                   # K_a = 2^64 - 3 meets K_b = 2 (over the wrap)
    wa[1], wb[1] = 3, 2
    wb[5] = (-(wa[4] + wa[7] + wb[9])) % M64
    wa[11] = (-(wb[12] + wb[13])) % M64
    W = 1 << logW
    if tr2:
        w2a = [rng.randrange(M64) for _ in range(na)]
        w2b = [rng.randrange(M64) for _ in range(nb)]
        W2 = 1 << 62
    else:
        w2a, w2b, W2 = [0] * na, [0] * nb, 0
    pairs = band_pairs_sorted(wa, wb, W)
    if tr2:
        a2, b2 = expand_values_u64(w2a), expand_values_u64(w2b)
        pairs = {(i, j) for (i, j) in pairs if accept((int(a2[i]) + int(b2[j])) % M64, M64, W2)}
    _PROD_CACHE[key] = (wa, wb, w2a, w2b, W, W2, pairs)
    return _PROD_CACHE[key]


@pytest.mark.parametrize("seed,na,nb,logW,tr2", [(61, 26, 27, 21, True), (62, 27, 27, 21, False)])
def test_match_fused_production_size_against_sorted_mitm(P, seed, na, nb, logW, tr2):
    """Completeness at the sizes the degree-100 problems run (2^26 + 2^27 and
    2^27 + 2^27 half-sums, 128 runs per half, 2^12 and 2^13 key units): the
    fused match's candidate set equals the oracle's sorted meet in the middle
    (every pair in the circular window, Eq. 9, then the Tr_2 test), with a
    window wide enough for thousands of pairs."""
    wa, wb, w2a, w2b, W, W2, pairs = _production_case(seed, na, nb, logW, tr2)
    assert len(pairs) >= 1000
    torch.cuda.empty_cache()
    got, ctr, raw = _run_match(P, wa, w2a, wb, w2b, W, W2, cap=1 << 16, fused=True)
    torch.cuda.empty_cache()
    assert ctr[4] == 0 and ctr[3] == 1
    assert len(raw) == len(set(raw)) == ctr[2]
    assert got == pairs - {(0, 0)}


def test_match_fused_32_element_halves_against_sorted_mitm(P):
    """Halves of 32 elements (2^32 + 2^32 half-sums, the degree-120 geometry:
    lists of 2^25 entries, 2^18 key units) whose top five weights are zero: the
    pair set is then exactly the oracle's pair set of the other 27 + 27
    elements times every choice of the zero elements (2^5 x 2^5), which the
    oracle computes by its sorted meet in the middle."""
    from oracle.recombine import accept, value
    wa27, wb27, _, _, _, _, wide = _production_case(62, 27, 27, 21, False)
    W = 1 << 10
    narrow = {(i, j) for (i, j) in wide
              if accept((value(i, wa27, M64) + value(j, wb27, M64)) % M64, M64, W)}
    wa, wb = wa27 + [0] * 5, wb27 + [0] * 5
    exp = {(i | (za << 27), j | (zb << 27)) for (i, j) in narrow for za in range(32) for zb in range(32)}
    assert len(narrow) >= 4 and len(exp) <= (1 << 17)
    torch.cuda.empty_cache()
    got, ctr, raw = _run_match(P, wa, [0] * 32, wb, [0] * 32, W, 0, cap=1 << 17, fused=True)
    torch.cuda.empty_cache()
    assert ctr[4] == 0 and ctr[3] == 1
    assert len(raw) == len(set(raw)) == ctr[2]
    assert got == exp - {(0, 0)}


def test_match_fused_clustered_keys_overflow(P):
    """2^15 keys of half a in one key unit overflow the fused table: the
    counters say so and the table match with the exact layout gives the scan."""
    from oracle.recombine import recombine_a
    rng = random.Random(78)
    na, nb = 15, 15
    wa = [rng.randrange(1 << 40) for _ in range(na)]
    wb = [rng.randrange(1 << 40) for _ in range(nb)]
    wa[0] = 0
    W = 1 << 20
    _, ctr, _ = _run_match(P, wa, [0] * na, wb, [0] * nb, W, 0, fused=True)
    assert ctr[4] == 1
    got, ctr2, _ = _run_match(P, wa, [0] * na, wb, [0] * nb, W, 0, exact=True)
    assert ctr2[4] == 0
    scan = set(recombine_a(wa + wb + [0], M64, W)) - {0}
    assert got == {(s & ((1 << na) - 1), s >> na) for s in scan} and (1, 0) in got


@pytest.mark.parametrize("seed,na,nb,compare_tables", [(41, 29, 30, True), (42, 30, 31, False)])
def test_match_fused_largest_halves(P, seed, na, nb, compare_tables):
    """The fused match at its largest halves (up to 2^10 runs per half, 2^30
    + 2^31 half-sums).  Every reported pair is re-checked one by one from its
    masks; the planted pairs (across the circular wrap, and three integral
    subsets) must all be found; at 2^29 + 2^30 the candidate set also equals
    the table match's (exact layout)."""
    from oracle.recombine import accept
    rng = random.Random(seed)
    wa = [rng.randrange(M64) for _ in range(na)]
    wb = [rng.randrange(M64) for _ in range(nb)]
    wa[0], wb[0] = M64 - 3, M64 - 2
    wa[1], wb[1] = 3, 2
    wb[5] = (-(wa[4] + wa[7] + wb[9])) % M64
    wa[11] = (-(wb[12] + wb[13])) % M64
    wb[20] = (-(wa[2] + wa[na - 1])) % M64
    W = 1 << 6                                        # about 2^(na+nb) * 2^7 / 2^64 random pairs
    torch.cuda.empty_cache()
    got, ctr, raw = _run_match(P, wa, [0] * na, wb, [0] * nb, W, 0, cap=1 << 16, fused=True)
    assert ctr[4] == 0 and ctr[3] == 1 and len(raw) == len(set(raw)) == ctr[2]
    for i, j in got:                                  # each reported pair, from its masks
        s = sum(wa[k] for k in range(na) if (i >> k) & 1) + sum(wb[k] for k in range(nb) if (j >> k) & 1)
        assert accept(s % M64, M64, W)
    planted = {(1, 0), (0, 1), (1 << 1, 1 << 1), (0, (1 << 5) | (1 << 9)), (1 << 11, (1 << 12) | (1 << 13)),
               ((1 << 4) | (1 << 7), (1 << 5) | (1 << 9)), ((1 << 2) | (1 << (na - 1)), 1 << 20)}
    planted = {(i, j) for i, j in planted
               if accept((sum(wa[k] for k in range(na) if (i >> k) & 1) +
                          sum(wb[k] for k in range(nb) if (j >> k) & 1)) % M64, M64, W)}
    assert len(planted) >= 5 and planted <= got
    if compare_tables:
        torch.cuda.empty_cache()
        got_t, ctr_t, _ = _run_match(P, wa, [0] * na, wb, [0] * nb, W, 0, cap=1 << 16, exact=True)
        assert ctr_t[4] == 0 and got_t == got
    torch.cuda.empty_cache()
