"""Write the golden factorisations under tests/golden/ by running the CPU oracle.

Every stored value comes from ``oracle.factor`` on inputs drawn by
``workloads``; nothing here touches the CUDA library.  Run from the repo root:

    python tests/golden/make_golden.py [--jobs 8] [--only cfg1,cfg2,...]

Files: ``<set>.json`` = a list of records
{name, seed, index, kind, coeffs, construction, factors, n, r, method,
 candidates (count), certificate_primes}.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SCAN_MAX_N = 33          # exhaustive RECOMBINE_A up to 2^32 patterns


def _special():
    from workloads import Instance, poly_mul
    def prod(fs):
        acc = [1]
        for f in fs:
            acc = poly_mul(acc, f)
        return acc
    out = []
    out.append(Instance([1, 0, -10, 0, 1], "special", None, tags={"name": "swinnerton_dyer_f2"}))
    out.append(Instance([576, 0, -960, 0, 352, 0, -40, 0, 1], "special", None, tags={"name": "swinnerton_dyer_f3"}))
    out.append(Instance(prod([[-i, 1] for i in range(1, 11)]), "special", [[-i, 1] for i in range(1, 11)], tags={"name": "linear_1_to_10"}))
    out.append(Instance([-1] + [0] * 11 + [1], "special", None, tags={"name": "x12_minus_1"}))
    out.append(Instance([-1] + [0] * 29 + [1], "special", None, tags={"name": "x30_minus_1"}))
    out.append(Instance([-1, -1, 0, 0, 0, 1], "special", None, tags={"name": "x5_minus_x_minus_1"}))
    out.append(Instance([1, 0, 0, 0, 1], "special", None, tags={"name": "x4_plus_1"}))
    out.append(Instance([-2, 1], "special", None, tags={"name": "linear"}))
    out.append(Instance([1, 1, 1], "special", None, tags={"name": "quadratic_pair"}))
    out.append(Instance(prod([[-2, 0, 1], [-3, 0, 1], [1, 1, 1]]), "special", None, tags={"name": "sqrt2_sqrt3_cyclo3"}))
    # close roots: +-sqrt(2000001) and +-sqrt(2000002) lie 3.5e-4 apart (2.5e-7 relative, a few
    # FP32 ulps), alone and beside a random degree-54 factor (about 32 elements: the fused match)
    import numpy as np
    from workloads import random_monic
    q1, q2 = [-2000001, 0, 1], [-2000002, 0, 1]
    f54 = random_monic(np.random.default_rng(20261204), 54, -100, 100)
    out.append(Instance(prod([q1, q2]), "special", [q1, q2], tags={"name": "close_quadratics"}))
    out.append(Instance(prod([q1, q2, f54]), "special", [q1, q2, f54], tags={"name": "close_quadratics_deg58"}))
    # Mignotte's x^16 - 2 (5x - 1)^2: two real roots near 1/5 about 5^-9 apart
    out.append(Instance([-2, 20, -50] + [0] * 13 + [1], "special", None, tags={"name": "mignotte_16"}))
    return out


def _sets(only):
    import workloads as W
    sets = {
        "cfg1": lambda: W.config1(1),
        "cfg2": lambda: W.config2(2),
        "cfg3": lambda: W.config3(3),
        "cfg4_sample": lambda: W.config4(4)[:64],
        "cfg5": lambda: W.config5(5),
        "special": _special,
    }
    return {k: v for k, v in sets.items() if not only or k in only}


def _one(args):
    name, inst = args
    from oracle import factor
    from oracle.zpoly import is_squarefree
    t0 = time.time()
    rec = {"name": inst.tags.get("name", f"{name}_{inst.index}"), "seed": inst.seed,
           "index": inst.index, "kind": inst.kind, "coeffs": inst.coeffs,
           "construction": inst.factors}
    if not is_squarefree(inst.coeffs):
        rec.update(error="not_squarefree")
        return rec
    res = factor(inst.coeffs, construction=inst.factors, max_scan_n=SCAN_MAX_N)
    rec.update(factors=res.factors, n=res.n, r=res.r, method=res.method,
               candidates=len(res.candidates), certificate_primes=res.certificate_primes,
               oracle_seconds=round(time.time() - t0, 3))
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    ap.add_argument("--only", default="")
    a = ap.parse_args()
    only = set(filter(None, a.only.split(",")))
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.jobs) as pool:
        for name, make in _sets(only).items():
            insts = make()
            t0 = time.time()
            recs = pool.map(_one, [(name, i) for i in insts], chunksize=1)
            with open(os.path.join(HERE, f"{name}.json"), "w") as f:
                json.dump(recs, f, indent=0)
            print(f"{name}: {len(recs)} records in {time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    main()
