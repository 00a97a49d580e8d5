"""Seeded synthetic workloads for the RFR hot path.

This module only draws integers and multiplies polynomials: it holds none of
the factorisation method's arithmetic.  The oracle (under ``oracle/``), the
tests and ``bench.py`` all take their inputs from here, so the CPU oracle and
the CUDA path always see the same polynomials for the same seed.

Polynomials are lists of Python ints in ascending powers, monic
(``p[-1] == 1``).  The shapes follow the workloads of Section 5 of the paper:
an input of degree d is the product of random monic polynomials whose
coefficients are uniform integers in a stated range; the coefficient range
applies to each factor, not to the product.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "Instance", "poly_mul", "random_monic", "random_composition",
    "product_instance", "random_instance", "config1", "config2", "config3",
    "config4", "config5", "random_weights",
]


@dataclass
class Instance:
    """One synthetic polynomial.

    ``coeffs``: ascending int coefficients, monic.  ``factors``: the random
    factors it was built from (None for a plain random polynomial).
    ``kind``: "product" or "random".  ``arrival_s``: request arrival time for
    serving workloads (None otherwise)."""
    coeffs: List[int]
    kind: str
    factors: Optional[List[List[int]]] = None
    seed: int = 0
    index: int = 0
    arrival_s: Optional[float] = None
    tags: dict = field(default_factory=dict)

    @property
    def degree(self) -> int:
        return len(self.coeffs) - 1


def poly_mul(a: List[int], b: List[int]) -> List[int]:
    """Exact product of two integer polynomials (ascending powers)."""
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return out


def random_monic(rng: np.random.Generator, degree: int, lo: int, hi: int) -> List[int]:
    """Monic polynomial of the given degree whose lower coefficients are
    uniform integers in [lo, hi].  The constant term is redrawn until it is
    non-zero, so that x never divides the result (products of such factors
    then stay square-free with overwhelming probability)."""
    if degree < 1:
        raise ValueError("degree must be >= 1")
    c = [int(v) for v in rng.integers(lo, hi + 1, size=degree)]
    while c[0] == 0:
        c[0] = int(rng.integers(lo, hi + 1))
    return c + [1]


def random_composition(rng: np.random.Generator, total: int, parts: int) -> List[int]:
    """Uniformly random composition of ``total`` into ``parts`` positive parts."""
    cuts = sorted(int(v) for v in rng.choice(np.arange(1, total), size=parts - 1, replace=False))
    edges = [0] + cuts + [total]
    return [edges[i + 1] - edges[i] for i in range(parts)]


def product_instance(rng, degrees, lo, hi, **kw) -> Instance:
    factors = [random_monic(rng, d, lo, hi) for d in degrees]
    p = [1]
    for f in factors:
        p = poly_mul(p, f)
    return Instance(coeffs=p, kind="product", factors=factors, **kw)


def random_instance(rng, degree, lo, hi, **kw) -> Instance:
    return Instance(coeffs=random_monic(rng, degree, lo, hi), kind="random", factors=None, **kw)


def config1(seed: int = 1) -> List[Instance]:
    """Degree 24: the product of two random degree-12 factors with
    coefficients in [-10, 10], plus one random degree-24 polynomial with
    coefficients in [-10, 10]."""
    rng = np.random.default_rng(seed)
    return [product_instance(rng, [12, 12], -10, 10, seed=seed, index=0),
            random_instance(rng, 24, -10, 10, seed=seed, index=1)]


def config2(seed: int = 2, count: int = 50) -> List[Instance]:
    """Degree 60 x ``count``: the first half products of 2-3 random factors
    (degree split a uniform composition of 60), the second half random;
    coefficients in [-100, 100]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if i < count // 2:
            k = int(rng.integers(2, 4))
            out.append(product_instance(rng, random_composition(rng, 60, k), -100, 100, seed=seed, index=i))
        else:
            out.append(random_instance(rng, 60, -100, 100, seed=seed, index=i))
    return out


def config3(seed: int = 3, count: int = 32) -> List[Instance]:
    """Degree 100 x ``count``: even indices are products (50+50, or a random
    3-part composition every fourth instance), odd indices random;
    coefficients in [-100, 100]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if i % 2 == 0:
            degs = [50, 50] if i % 4 == 0 else random_composition(rng, 100, 3)
            out.append(product_instance(rng, degs, -100, 100, seed=seed, index=i))
        else:
            out.append(random_instance(rng, 100, -100, 100, seed=seed, index=i))
    return out


def config4(seed: int = 4, count: int = 10000, rate_per_s: float = 100.0,
            dmin: int = 20, dmax: int = 100) -> List[Instance]:
    """Serving stream: degrees uniform in [dmin, dmax], coefficients in
    [-1000, 1000], 30 % products of 2-3 random factors; Poisson arrivals at
    ``rate_per_s`` (exponential inter-arrival gaps), stored in ``arrival_s``."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for i in range(count):
        d = int(rng.integers(dmin, dmax + 1))
        t += float(rng.exponential(1.0 / rate_per_s))
        if rng.random() < 0.3:
            k = int(rng.integers(2, 4))
            inst = product_instance(rng, random_composition(rng, d, k), -1000, 1000, seed=seed, index=i)
        else:
            inst = random_instance(rng, d, -1000, 1000, seed=seed, index=i)
        inst.arrival_s = t
        out.append(inst)
    return out


def config5(seed: int = 5) -> List[Instance]:
    """Degree 120: the product of two random degree-60 factors with
    coefficients in [-100, 100]."""
    rng = np.random.default_rng(seed)
    return [product_instance(rng, [60, 60], -100, 100, seed=seed, index=0)]


def random_weights(seed: int, count: int) -> np.ndarray:
    """Uniform random 64-bit weights (uint64) for stage-level tests of the
    enumeration and match kernels."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**64, size=count, dtype=np.uint64)
