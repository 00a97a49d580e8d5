"""Algorithm B (Section 3.2) on the GPU against the oracle's RECOMBINE_B and
the sorted meet in the middle; the runtime with rfr_config.match_path =
RFR_MATCH_PRUNE against the goldens."""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import golden, to_u64, u64_tensor  # noqa: E402
from oracle.prune import improvement_ratio, recombine_b  # noqa: E402
from oracle.recombine import band_pairs_sorted, expand_values  # noqa: E402

M64 = 1 << 64


@pytest.fixture(scope="module")
def P():
    import paper_2410_15880_b300 as P
    return P


def _prune(P, w, w2, W, W2, cap=1 << 20):
    m = len(w)
    cand, ctr, _ = P.stage_prune(u64_tensor(w or [0])[:m], u64_tensor(w2 or [0])[:m], W, W2, cap)
    torch.cuda.synchronize()
    c = [int(x) for x in to_u64(ctr)]
    return {int(x) for x in to_u64(cand)[:min(c[2], cap)]}, c


@pytest.mark.parametrize("m,shift", [(0, 2), (1, 2), (10, 4), (14, 9), (20, 14), (22, 16)])
def test_prune_equals_oracle(P, m, shift):
    rng = random.Random(m + 3)
    w = [rng.randrange(M64) for _ in range(m)]
    if m >= 6:
        w[4] = (-(w[1] + w[5])) % M64
    W = M64 >> shift
    acc, visited, _ = recombine_b(w, M64, W)
    got, c = _prune(P, w, [0] * m, W, 0)
    assert c[3] == 1 and c[1] == len(acc)
    assert got == set(acc) - {0} and c[2] == len(got)
    assert c[0] >= visited                       # blocks of 2^B patterns: jumps never leave a block


def test_prune_tr2(P):
    rng = random.Random(5)
    m = 12
    w = [rng.randrange(M64) for _ in range(m)]
    w2 = [rng.randrange(M64) for _ in range(m)]
    W, W2 = M64 >> 5, M64 >> 2
    acc = set(recombine_b(w, M64, W)[0]) - {0}
    t2 = expand_values(w2, M64)
    exp = {s for s in acc if min(t2[s], M64 - t2[s]) <= W2}
    got, c = _prune(P, w, w2, W, W2)
    assert 0 < len(exp) < len(acc) and got == exp


@pytest.mark.parametrize("m", [28, 32])
def test_prune_large_against_sorted_mitm(P, m):
    """m = 28 and 32 (2^28, 2^32 patterns; threads walk 2^8, 2^12): the
    accepted set equals the sorted meet in the middle's, and the pruning
    visits a fraction of the patterns near Theorem 3.2.1's estimate."""
    rng = random.Random(m)
    w = [rng.randrange(M64) for _ in range(m)]
    w[7] = (-(w[0] + w[20] + w[3])) % M64
    W = M64 >> (m + 6)
    h = m // 2
    exp = {a | (b << h) for a, b in band_pairs_sorted(w[:h], w[h:], W)} - {0}
    got, c = _prune(P, w, [0] * m, W, 0)
    assert (1 | 1 << 3 | 1 << 7 | 1 << 20) in exp
    assert got == exp
    ratio = (1 << m) / c[0]
    print(f"m={m}: visited {c[0]} of 2^{m} patterns, ratio {ratio:.1f}, Theorem 3.2.1 {improvement_ratio(m):.1f}")
    assert ratio > 0.25 * improvement_ratio(m)


def test_factor_prune_path_equals_goldens(P):
    """Problems of at most 40 searched elements through Algorithm B, the rest
    through the automatic choice: the goldens' factorisations."""
    recs = golden("cfg2")[:10] + golden("cfg1") + golden("special") + golden("cfg3")[:2]
    with P.Context(device=0, match_path=P.RFR_MATCH_PRUNE) as c:
        res = c.factor_batch([r["coeffs"] for r in recs])
    for r, x in zip(recs, res):
        assert x.ok and x.factors == r["factors"], r.get("name")
