"""End-to-end parity: rfr_factor / rfr_factor_batch / serving against the
oracle's golden factorisations (bit-exact canonical factor lists)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import golden  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_2410_15880_b300 import Context
    c = Context(device=0, timing=True)
    yield c
    c.close()


def check_batch(ctx, recs):
    res = ctx.factor_batch([r["coeffs"] for r in recs])
    bad = [(r["name"], x.status, x.factors, r["factors"]) for r, x in zip(recs, res)
           if not (x.ok and x.factors == r["factors"])]
    assert not bad, bad[:3]
    for r, x in zip(recs, res):
        if "n" in r and r["n"] > 1:
            assert x.diag["n"] == r["n"] and x.diag["r"] == r["r"], r["name"]
        if len(r["coeffs"]) > 2:
            assert 0.0 < x.diag["max_rel_residual"] <= 1e-10, (r["name"], x.diag["max_rel_residual"])
    return res


def test_single_degree24(ctx):
    for r in golden("cfg1"):
        x = ctx.factor(r["coeffs"])
        assert x.ok and x.factors == r["factors"]


def test_special_polynomials(ctx):
    res = check_batch(ctx, golden("special"))
    sd = [x for r, x in zip(golden("special"), res) if r["name"] == "swinnerton_dyer_f2"][0]
    assert sd.diag["cand_pre"] >= 1 and sd.diag["verified"] == 0     # false candidates rejected


def test_degree60_batch(ctx):
    check_batch(ctx, golden("cfg2"))


def test_serving_sample_batch(ctx):
    check_batch(ctx, golden("cfg4_sample"))


def test_degree100_batch(ctx):
    res = check_batch(ctx, golden("cfg3"))
    assert all(x.diag["half_sums"] > (1 << 24) for x in res)


def test_degree100_batch_fp64_roots():
    from paper_2410_15880_b300 import Context, RFR_ROOTS_FP64
    with Context(device=0, root_mode=RFR_ROOTS_FP64) as c:
        res = check_batch(c, golden("cfg3")[:16] + golden("cfg2")[:8])
    assert all(x.diag["max_root_err"] < 1e-20 for x in res)


def test_degree120_product(ctx):
    res = check_batch(ctx, golden("cfg5"))
    assert res[0].diag["n_b"] >= 30 and res[0].diag["half_sums"] > (1 << 31)


def test_one_launch_per_polynomial_equals_batch(ctx):
    recs = golden("cfg2")[:8]
    batch = ctx.factor_batch([r["coeffs"] for r in recs])
    for r, b in zip(recs, batch):
        a = ctx.factor(r["coeffs"])
        assert a.factors == b.factors == r["factors"]


def test_error_statuses(ctx):
    from paper_2410_15880_b300._native import status_name
    cases = {
        "RFR_E_NOT_MONIC": [1, 2, 3],
        "RFR_E_RANGE": [1 << 60, 1],
        "RFR_E_NOT_SQUAREFREE": [2, -3, 0, 1],            # (x-1)^2 (x+2)
    }
    for want, p in cases.items():
        assert status_name(ctx.factor(p).status) == want
    assert ctx.factor([-7, 1]).factors == [[-7, 1]]      # degree 1
    assert ctx.factor([1, 0, 0, 0, 1]).factors == [[1, 0, 0, 0, 1]]    # x^4+1 irreducible over Z


def test_root_cluster_below_fp64_resolution_is_reported():
    """x^24 - 2 (5x - 1)^2 (Mignotte) has two real roots near 1/5 about 1.6e-9
    apart, closer than its FP64 root finder can resolve them (its error there is
    about 1e-16 |p| / |p'|, near 1e-6), so the inclusion discs cannot be
    separated: the call must then report RFR_E_ROOTS, never a wrong list (it is
    irreducible, which the oracle proves; this build reports RFR_E_ROOTS).  Two
    roots 3.5e-4 apart at 1414 (the special goldens close_quadratics*) are
    resolved by the further double-double Newton steps."""
    from paper_2410_15880_b300 import Context
    from paper_2410_15880_b300._native import status_name
    p = [-2, 20, -50] + [0] * 21 + [1]
    with Context(device=0) as c:
        x = c.factor(p)
    assert (x.ok and x.factors == [p]) or (status_name(x.status) == "RFR_E_ROOTS" and not x.factors)


def test_serving_alone_and_in_mix():
    from paper_2410_15880_b300 import Context
    recs = golden("cfg4_sample")
    with Context(device=0, max_inflight=2, max_batch=16) as srv:
        tickets = [srv.submit(r["coeffs"]) for r in recs]
        out = [srv.wait(t, 120000) for t in tickets]
        alone = srv.factor(recs[5]["coeffs"])
    for r, x in zip(recs, out):
        assert x.ok and x.factors == r["factors"], r["name"]
    # batches formed from the request queue launch directly: no graph is captured on the request path
    assert all(x.diag["graphs"] == 0 for x in out)
    mixed = out[5]
    assert alone.factors == mixed.factors
    assert alone.diag["n"] == mixed.diag["n"] and alone.diag["window"] == mixed.diag["window"]


def test_serving_cancel_and_poll():
    from paper_2410_15880_b300 import Context
    recs = golden("cfg2")[:20]
    with Context(device=0, max_inflight=1, max_batch=1) as srv:
        ts = [srv.submit(r["coeffs"]) for r in recs]
        last = ts[-1]
        st = srv.cancel(last)
        assert st in (0, 1)                      # cancelled while queued, or already running
        for t, r in zip(ts[:-1], recs[:-1]):
            x = srv.wait(t, 120000)
            assert x.factors == r["factors"]
        x = srv.wait(last, 120000)
        assert x.status in (0, -14)
        assert srv.cancel(10 ** 9) == -1        # unknown ticket


def test_device_input_batch(ctx):
    import numpy as np
    recs = golden("cfg2")[:10] + golden("special")
    arr = np.zeros((len(recs), 129), dtype=np.int64)
    for i, r in enumerate(recs):
        arr[i, :len(r["coeffs"])] = r["coeffs"]
    d_co = torch.from_numpy(arr).cuda()
    d_dg = torch.tensor([len(r["coeffs"]) - 1 for r in recs], dtype=torch.int32, device="cuda")
    res = ctx.factor_batch_device(d_co, d_dg)
    for r, x in zip(recs, res):
        assert x.ok and x.factors == r["factors"], r["name"]
    assert res[0].diag["batch_size"] == len(recs) and res[0].diag["launches"] >= 5


def test_device_input_checks(ctx):
    import numpy as np
    from paper_2410_15880_b300._native import status_name
    polys = [[1, 2, 3], [1 << 60, 1], [2, -3, 0, 1], [-7, 1], [1, 0, 0, 0, 1]]
    arr = np.zeros((len(polys), 129), dtype=np.int64)
    for i, p in enumerate(polys):
        arr[i, :len(p)] = p
    res = ctx.factor_batch_device(torch.from_numpy(arr).cuda(),
                                  torch.tensor([len(p) - 1 for p in polys], dtype=torch.int32, device="cuda"))
    assert [status_name(x.status) for x in res[:3]] == ["RFR_E_NOT_MONIC", "RFR_E_RANGE", "RFR_E_NOT_SQUAREFREE"]
    assert res[3].factors == [[-7, 1]] and res[4].factors == [[1, 0, 0, 0, 1]]


def test_validate_stage_suspect_then_roots_decide(ctx):
    from gpu_util import coeff_tensor
    import paper_2410_15880_b300 as P
    # square-free, but its discriminant is divisible by neither Mersenne prime: proven OK
    c, d = coeff_tensor([[1, 0, -10, 0, 1], [2, -3, 0, 1]])
    st = P.stage_validate(c, d).cpu().tolist()
    assert st == [0, 2]                       # (x-1)^2 (x+2): gcd(p, p') = x-1 modulo every prime


def test_autotune_and_graphs_do_not_change_results(tmp_path):
    from paper_2410_15880_b300 import Context
    recs = golden("cfg2")[:12] + golden("cfg3")[:4]
    cache = str(tmp_path / "tune.txt")
    with Context(device=0, autotune=True, tune_cache_path=cache) as c:
        check_batch(c, recs)
        check_batch(c, recs)                       # second pass uses the cache and the captured graph
    lines = open(cache).read().strip().splitlines()
    assert len(lines) >= 2 and all(len(l.split("\t")[1].split()) == 7 for l in lines)
    with Context(device=0, use_graphs=False, tune_cache_path=cache) as c:
        check_batch(c, recs)


def test_match_graph_captured_on_second_occurrence_and_replayed():
    """A batch whose problems all take the fused match: the first call launches
    the match directly, the second captures its launch shape as a CUDA graph,
    the third replays it.  Every call returns the goldens with the same
    candidate counts, the stage timings recorded by the graph's event nodes are
    positive, and a batch of another shape in between does not disturb it.
    Small problems (the shared-memory match) are captured and replayed the
    same way."""
    import numpy as np
    import torch
    from paper_2410_15880_b300 import Context
    recs = golden("cfg3")[:3] + golden("cfg2")[:5]
    other = golden("cfg2")[5:9]
    arr = np.zeros((len(recs), 129), dtype=np.int64)
    for i, r in enumerate(recs):
        arr[i, :len(r["coeffs"])] = r["coeffs"]
    d_co = torch.from_numpy(arr).cuda()
    d_dg = torch.tensor([len(r["coeffs"]) - 1 for r in recs], dtype=torch.int32, device="cuda")
    with Context(device=0, timing=True) as c:
        runs = []
        for k in range(3):
            runs.append(c.factor_batch_device(d_co, d_dg))
            if k == 1:
                check_batch(c, other)
    with Context(device=0, timing=True) as c:
        host = [check_batch(c, recs) for _ in range(3)]
        small = golden("cfg1")
        assert all(r["n"] - 1 <= 26 for r in small)                 # halves of <= 13: the shared-memory match
        tiny = [check_batch(c, small) for _ in range(3)]
    assert [runs[k][0].diag["graphs"] for k in range(3)] == [0, 1, 1]
    assert [host[k][0].diag["graphs"] for k in range(3)] == [1, 2, 2]     # prologue graph + match graph
    assert [tiny[k][0].diag["graphs"] for k in range(3)] == [1, 2, 2]     # prologue graph + k_small graph
    for res in runs + host:
        assert [x.factors for x in res] == [r["factors"] for r in recs]
        assert [x.diag["cand_post"] for x in res] == [x.diag["cand_post"] for x in runs[0]]
    for res in (runs[2], host[2]):
        st = res[0].diag["stage_us"]
        assert st[2] > 0 and st[4] > 0, list(st)           # sorted lists; match (event nodes of the graph)
    assert host[2][0].diag["stage_us"][0] > 0                # roots (event nodes of the prologue graph)


def test_every_fused_layout_the_tuner_may_keep_gives_the_same_results(tmp_path):
    """Each fused-match layout the autotuner times (key units of 2^12, 2^13 or
    2^14 half-a keys, at most 2^12 or 2^13 bins per unit), forced through a
    tune cache file, returns the goldens with the same exact candidate counts
    as the default layout: the candidates are the pairs in the window, however
    the key space is tiled."""
    import torch
    from paper_2410_15880_b300 import Context
    recs = golden("cfg3")[:4] + golden("cfg2")[:8] + golden("cfg5")
    with Context(device=0) as c:
        base = check_batch(c, recs)
    classes = sorted({(x.diag["n_a"], x.diag["n_b"]) for x in base if x.diag["n_a"] >= 14})
    assert len(classes) >= 3
    dev = torch.cuda.get_device_name(0)
    for ulog, nbl in [(13, 13), (12, 13), (14, 12), (12, 12)]:
        path = tmp_path / f"tune_{ulog}_{nbl}.txt"
        path.write_text("".join(f"{dev}\t{na} {nb} 16 13 16 {ulog} {nbl}\n" for na, nb in classes))
        with Context(device=0, tune_cache_path=str(path)) as c:
            res = check_batch(c, recs)
        assert [x.diag["cand_pre"] for x in res] == [x.diag["cand_pre"] for x in base], (ulog, nbl)
        assert [x.diag["cand_post"] for x in res] == [x.diag["cand_post"] for x in base], (ulog, nbl)


def test_tables_only_equals_fused():
    """The same batch through the table match only (rfr_config.match_path =
    RFR_MATCH_TABLES) and through the automatic choice (the fused match for
    these sizes): identical factorisations, equal to the oracle's goldens."""
    from paper_2410_15880_b300 import Context
    recs = golden("cfg3")[:6] + golden("cfg2")[:8]
    polys = [r["coeffs"] for r in recs]
    with Context(device=0) as auto, Context(device=0, tables_only=True) as tab:
        ra = auto.factor_batch(polys)
        rt = tab.factor_batch(polys)
    for r, a, t in zip(recs, ra, rt):
        assert a.ok and t.ok
        assert a.factors == t.factors == r["factors"]
        assert a.diag["cand_post"] == t.diag["cand_post"]


def _run_shards(polys, nshards, timeout=600.0):
    """factor_batch_sharded for every shard, one thread and context each, the
    verified sets exchanged on the host.  The exchange gives up well before
    the join limit, so a stuck shard ends with its own error; every shard's
    exception is re-raised here, and no shard is left running."""
    import threading
    from paper_2410_15880_b300 import Context
    from paper_2410_15880_b300.sharding import ThreadExchange
    ex = ThreadExchange(nshards, timeout=timeout / 4)
    out, err = [None] * nshards, [None] * nshards

    def run(s):
        try:
            with Context(device=0, mem_budget_bytes=16 << 30) as c:
                out[s] = c.factor_batch_sharded(polys, s, nshards, ex.gather_for(s))
        except BaseException as e:                     # noqa: BLE001 - handed to the test thread
            err[s] = e
    th = [threading.Thread(target=run, args=(s,)) for s in range(nshards)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=timeout)
    assert not any(t.is_alive() for t in th), "a shard did not finish"
    for e in err:
        if e is not None:
            raise e
    return out


def test_key_range_shards_equal_whole_batch():
    """Two key-range shards of one batch, run by two threads with their own
    contexts on this GPU and exchanging verified sets on the host (no kernel
    waits on another): both return the goldens' factorisations, and the fused
    problems' candidates split between the shards without overlap."""
    from paper_2410_15880_b300 import Context
    recs = golden("cfg3")[:4] + golden("cfg2")[:4] + golden("cfg1") + golden("special")
    polys = [r["coeffs"] for r in recs]
    with Context(device=0, mem_budget_bytes=16 << 30) as c:
        whole = c.factor_batch(polys)
    out = _run_shards(polys, 2)
    for r, w, a, b in zip(recs, whole, out[0], out[1]):
        assert w.ok and a.ok and b.ok, r.get("name")
        assert a.factors == b.factors == w.factors == r["factors"]
        if w.diag["n_a"] >= 14:                       # fused: the shards partition the key units
            assert a.diag["cand_post"] + b.diag["cand_post"] == w.diag["cand_post"]
        else:                                         # small halves: matched on shard 0
            assert b.diag["cand_post"] == 0


def test_poll_batch_serving():
    """rfr_poll_batch: many requests tracked with one call per sweep; every
    result equals its golden and each ticket is released once."""
    import time
    from paper_2410_15880_b300 import Context
    recs = golden("cfg4_sample")[:24] + golden("cfg2")[:8]
    with Context(device=0, max_inflight=2, max_batch=16) as c:
        tickets = [c.submit(r["coeffs"]) for r in recs]
        results, pending = {}, list(range(len(recs)))
        deadline = time.time() + 120
        while pending and time.time() < deadline:
            got = c.poll_batch([tickets[i] for i in pending])
            pending = [i for i, r in zip(pending, got) if r is None or results.setdefault(i, r) is None]
            time.sleep(0.001)
        assert not pending
        assert all(results[i].ok and results[i].factors == r["factors"] for i, r in enumerate(recs))
        again = c.poll_batch(tickets[:3])                  # released tickets are unknown now
        assert all(x is not None and x.status == -1 for x in again)


def test_key_range_shards_with_table_redo():
    """x^60 - 1 (clustered keys: the fused match overflows and the problem is
    redone whole with the table match) plus a degree-100 golden, in two
    key-range shards: both shards return the cyclotomic factors and the
    golden, the same as the unsharded batch."""
    from oracle import canonical
    from test_oracle_pins import cyclotomic
    m = 60
    polys = [[-1] + [0] * (m - 1) + [1], golden("cfg3")[0]["coeffs"]]
    expect = [canonical([cyclotomic(k) for k in range(1, m + 1) if m % k == 0]), golden("cfg3")[0]["factors"]]
    out = _run_shards(polys, 2)
    for s in range(2):
        assert [r.ok for r in out[s]] == [True, True], [r.status for r in out[s]]
        assert [r.factors for r in out[s]] == expect


def test_async_batches_in_flight_equal_golden():
    """rfr_factor_batch_async: three batches queued back to back (two run at
    once on the two workers) give the golden factorisations, error statuses
    included, whatever order they are waited in; result() is idempotent."""
    from paper_2410_15880_b300 import Context
    from paper_2410_15880_b300._native import status_name
    recs2, recs3 = golden("cfg2")[:20], golden("cfg3")[:6]
    bad = [[1, 2, 3], [1 << 60, 1], [2, -3, 0, 1], [5]]   # not monic, range, not square-free, degree 0
    want_bad = ["RFR_E_NOT_MONIC", "RFR_E_RANGE", "RFR_E_NOT_SQUAREFREE", "RFR_E_RANGE"]
    with Context(device=0, max_inflight=2) as c:
        h1 = c.factor_batch_async([r["coeffs"] for r in recs2])
        h2 = c.factor_batch_async([r["coeffs"] for r in recs3] + bad)
        h3 = c.factor_batch_async([r["coeffs"] for r in recs2[::-1]])
        r3, r1, r2 = h3.result(), h1.result(), h2.result()
        assert h1.result() is r1
        sync = c.factor_batch([r["coeffs"] for r in recs3])
        assert c.factor_batch_async([]).result() == []
    assert [x.factors for x in r1] == [r["factors"] for r in recs2] and all(x.ok for x in r1)
    assert [x.factors for x in r3] == [r["factors"] for r in recs2[::-1]]
    assert [x.factors for x in r2[:6]] == [r["factors"] for r in recs3] == [x.factors for x in sync]
    assert [status_name(x.status) for x in r2[6:]] == want_bad
    assert r2[0].diag["n"] == sync[0].diag["n"] and r2[0].diag["window"] == sync[0].diag["window"]


def test_async_wait_unknown_ticket_and_destroy_with_queued_batches():
    """rfr_batch_wait on an unknown ticket is RFR_E_INVALID; rfr_destroy with
    batches still queued drops them (statuses RFR_E_CANCELLED, outs zeroed)
    and lets the running ones finish (their results are the caller's)."""
    import ctypes as C
    from paper_2410_15880_b300._native import Config, Factors, lib, _marshal
    L = lib()
    cfg = Config()
    assert L.rfr_config_default(C.byref(cfg)) == 0
    cfg.device, cfg.max_inflight = 0, 1
    h = C.c_void_p()
    assert L.rfr_create(C.byref(cfg), C.byref(h)) == 0
    assert L.rfr_batch_wait(h, 12345, 0) == -1
    recs = golden("cfg2")[:10]
    keep, jobs = [], []
    for _ in range(6):
        n, ptrs, degs, k = _marshal([r["coeffs"] for r in recs])
        outs, sts, t = (Factors * n)(), (C.c_int * n)(), C.c_uint64(0)
        assert L.rfr_factor_batch_async(h, n, ptrs, degs, outs, sts, C.byref(t)) == 0
        keep.append(k)
        jobs.append((outs, sts, n))
    assert L.rfr_destroy(h) == 0
    cancelled = 0
    for outs, sts, n in jobs:
        st = list(sts)
        if st == [-14] * n:
            cancelled += 1
            assert all(outs[i].n_factors == 0 for i in range(n))
        else:
            assert st == [0] * n
        L.rfr_factors_free_n(outs, n)
    assert 0 <= cancelled <= 6


def test_async_handles_dropped_or_waited_after_close():
    """A handle dropped before its result() leaves the result arrays with the
    context (the workers still write into them), which releases them at
    close(); result() after close() raises instead of touching freed state."""
    import gc
    from paper_2410_15880_b300 import Context, RFRError
    recs = golden("cfg2")[:10]
    polys = [r["coeffs"] for r in recs]
    c = Context(device=0, max_inflight=2)
    for _ in range(4):
        c.factor_batch_async(polys)               # handle dropped at once
    gc.collect()
    kept = c.factor_batch_async(polys)
    assert [x.factors for x in kept.result()] == [r["factors"] for r in recs]
    late = c.factor_batch_async(polys)
    c.close()
    with pytest.raises(RFRError):
        late.result()
    assert [x.factors for x in kept.result()] == [r["factors"] for r in recs]   # already taken
