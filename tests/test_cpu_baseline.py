"""The multithreaded CPU Horowitz–Sahni baseline against the oracle's pair
sets (brute force, and the sorted meet in the middle for larger halves)."""
import random

import pytest

from oracle.recombine import band_pairs, band_pairs_sorted, expand_values

M64 = 1 << 64


@pytest.fixture(scope="module")
def hs():
    import baseline
    baseline.build()
    return baseline


def _pairs(cands, n_a):
    return {(c & ((1 << n_a) - 1), c >> n_a) for c in cands}


@pytest.mark.parametrize("n_a,n_b,threads", [(0, 1, 1), (3, 4, 2), (7, 8, 3), (9, 10, 8)])
def test_matches_brute_force(hs, n_a, n_b, threads):
    rng = random.Random(n_a * 31 + n_b)
    wa = [rng.randrange(M64) for _ in range(n_a)]
    wb = [rng.randrange(M64) for _ in range(n_b)]
    if n_a >= 2:
        wb[0] = (-(wa[0] + wa[1])) % M64                  # a planted integral pair
    W = M64 >> 8 if n_a + n_b > 10 else M64 >> 3       # wide: many pairs, windows that wrap
    exp = band_pairs(expand_values(wa, M64), expand_values(wb, M64), M64, W)
    z = [0] * max(n_a, n_b)
    cands, counts, _ = hs.hs_mt_match(wa, z[:n_a], wb, z[:n_b], W, 0, threads=threads, cap=1 << 20)
    assert counts[0] == len(exp) and counts[2] == 1
    assert _pairs(cands, n_a) == exp - {(0, 0)}
    assert len(cands) == counts[1]


def test_tr2_prefilter(hs):
    """Candidates are the pairs within W whose w2 sums are within W2."""
    rng = random.Random(7)
    wa = [rng.randrange(M64) for _ in range(8)]
    wb = [rng.randrange(M64) for _ in range(9)]
    w2a = [rng.randrange(M64) for _ in range(8)]
    w2b = [rng.randrange(M64) for _ in range(9)]
    W, W2 = M64 >> 6, M64 >> 2
    pairs = band_pairs(expand_values(wa, M64), expand_values(wb, M64), M64, W) - {(0, 0)}
    t2a, t2b = expand_values(w2a, M64), expand_values(w2b, M64)
    exp = {(i, j) for i, j in pairs if min((t2a[i] + t2b[j]) % M64, (-(t2a[i] + t2b[j])) % M64) <= W2}
    assert 0 < len(exp) < len(pairs)
    cands, counts, _ = hs.hs_mt_match(wa, w2a, wb, w2b, W, W2, threads=4, cap=1 << 20)
    assert _pairs(cands, 8) == exp and counts[0] == len(pairs) + 1


def test_larger_halves_against_sorted_mitm(hs):
    rng = random.Random(11)
    wa = [rng.randrange(M64) for _ in range(14)]
    wb = [rng.randrange(M64) for _ in range(15)]
    W = M64 >> 20                                      # about 2^29 * 2^-19 = 1000 pairs
    exp = band_pairs_sorted(wa, wb, W)
    cands, counts, secs = hs.hs_mt_match(wa, [0] * 14, wb, [0] * 15, W, 0, cap=1 << 20)
    assert _pairs(cands, 14) == exp - {(0, 0)} and counts[0] == len(exp)
    assert len(secs) == 3 and all(s >= 0 for s in secs)


def test_rejects_bad_arguments(hs):
    with pytest.raises(ValueError):
        hs.hs_mt_match([1] * 33, [0] * 33, [1], [0], 10, 0)
    with pytest.raises(ValueError):
        hs.hs_mt_match([1], [0], [1], [0], 1 << 63, 0)


@pytest.mark.parametrize("n_a,n_b,logW,threads", [(16, 16, 30, 3), (17, 18, 36, 8), (20, 21, 24, 16)])
def test_runs_design_against_sorted_mitm(hs, n_a, n_b, logW, threads):
    """Halves of 16 elements and more take the runs design (sorted low lists,
    runs, key units, binned half a): its pair set is the oracle's, with pairs
    planted across the circular wrap and integral subsets."""
    rng = random.Random(n_a * 7 + n_b)
    wa = [rng.randrange(M64) for _ in range(n_a)]
    wb = [rng.randrange(M64) for _ in range(n_b)]
    wa[0], wb[0] = M64 - 3, M64 - 2                    # K_a = 2^64 - 3 meets K_b = 2 (over the wrap)
    wa[1], wb[1] = 3, 2
    wb[5] = (-(wa[4] + wa[7] + wb[9])) % M64
    wa[n_a - 1] = (-(wb[n_b - 1] + wb[12])) % M64     # a high element of each half
    W = 1 << logW
    exp = band_pairs_sorted(wa, wb, W)
    cands, counts, secs = hs.hs_mt_match(wa, [0] * n_a, wb, [0] * n_b, W, 0, threads=threads, cap=1 << 20)
    assert secs[1] == 0.0                              # no sort: the runs design ran
    assert counts[0] == len(exp) and counts[2] == 1
    assert _pairs(cands, n_a) == exp - {(0, 0)}
