"""rfr_factor_general on the GPU: any nonzero p in Z[x] (content, powers of
x, multiplicities, non-monic factors) against constructions with known
irreducible factors and the oracle's factor_general."""
import json
import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.squarefree import expand, factor_general  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def canon(fs):
    return sorted(fs, key=lambda fm: (len(fm[0]) - 1, tuple(fm[0]), fm[1]))


@pytest.fixture(scope="module")
def ctx():
    import paper_2410_15880_b300 as P
    with P.Context(device=0) as c:
        yield c


def golden(name):
    return json.load(open(os.path.join(HERE, "golden", f"{name}.json")))


EIS = [[1, 2], [-2, 0, 3], [3, 3, 0, 5], [3, 3, 0, 0, 7]]     # Eisenstein at 2, 2, 3, 3 (irreducible)


def test_constructions(ctx):
    monic = [f for r in golden("cfg1") for f in r["factors"] if len(f) > 2][:2]
    cases = [(-6, [(EIS[0], 2), (EIS[1], 1), ([0, 1], 3)]),
             (1, [(monic[0], 2), (EIS[2], 1)]),
             (5, [(EIS[1], 3), ([-1, 1], 1), ([1, 1], 2)]),
             (-1, [(EIS[3], 1), (EIS[2], 2), ([1, 0, 1], 2)]),
             (2, [(monic[0], 1), (monic[1], 1), ([0, 1], 1)])]
    for c, fs in cases:
        p = expand(c, fs)
        r = ctx.factor_general(p)
        assert r.ok, (p, r.status)
        assert r.content == c and r.factors == canon(fs)
        assert (r.content, r.factors) == factor_general(p)


def test_degree60_with_content(ctx):
    """2 p for degree-60 inputs with goldens: one square-free part, factored
    by the fused match."""
    for rec in golden("cfg2")[:4]:
        p = [2 * x for x in rec["coeffs"]]
        r = ctx.factor_general(p)
        assert r.ok and r.content == 2
        assert r.factors == [(f, 1) for f in rec["factors"]]


def test_edge_cases(ctx):
    assert ctx.factor_general([0, 0]).status == -1                 # the zero polynomial
    r = ctx.factor_general([-7])
    assert r.ok and r.content == -7 and r.factors == []
    r = ctx.factor_general([0, 0, 0, 4])                           # 4 x^3
    assert r.ok and r.content == 4 and r.factors == [([0, 1], 3)]
    big = [1] * 20 + [1000]                                        # lc^19 > 2^53 after the transform
    assert ctx.factor_general(big).status == -3
