"""Benchmark of the RFR hot path on B300 (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config cfg3|cfg2|cfg1|cfg5] [--count C] [--no-cpu-baseline]

A step factors one batch of synthetic polynomials end to end (validate,
roots, weights, enumerate + radix partition, match, verify, atoms).  The
default workload is 32 polynomials of degree 100, coefficients uniform in
[-100, 100], half products of random factors and half random (seed 3 + 1000
* rank).  `value` is polynomials/s with the coefficients already in device
memory (rfr_factor_batch_device), one blocking call per step; `e2e` is the
same from host buffers through rfr_factor_batch_async with four batches in
flight (the blocking rfr_factor_batch is reported beside it).  Under torchrun each rank runs its own batch on its own GPU
(weak scaling, no data-path collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "polynomials factored/sec at degree 100 (32-polynomial batch)"
UNIT = "polys/s"
E2E_DEPTH = 4            # batches in flight in the end-to-end leg (worker pipelines of its context)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cfg3", choices=["cfg1", "cfg2", "cfg3", "cfg5"])
    ap.add_argument("--count", type=int, default=0, help="use only the first C polynomials")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=10000,
                    help="requests of the serving stream (0 = skip the serving leg)")
    ap.add_argument("--serving-loads", default="0.5,0.8,0.95",
                    help="Poisson arrival rates as fractions of the measured closed-loop capacity")
    ap.add_argument("--serving-trace", default="",
                    help="write per-request arrival/submit/done times to PATH.load<L>.csv")
    ap.add_argument("--root-mode", type=int, default=1,
                    help="0 = FP64 Aberth, 1 = FP32 bulk + FP64 (default)")
    ap.add_argument("--no-autotune", action="store_true", help="use the default match layout")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the prologue and the match directly instead of replaying captured graphs")
    ap.add_argument("--match-path", default="auto", choices=["auto", "tables", "splat", "prune"],
                    help="rfr_config.match_path: automatic choice, table match only, the splat match "
                         "(Algorithm E) or the pruned search (Algorithm B)")
    ap.add_argument("--tune-cache", default="", help="file that stores tuned match layouts")
    ap.add_argument("--degree60-steps", type=int, default=40,
                    help="steps of the degree-60 sub-measurement (0: skip)")
    ap.add_argument("--degree120-steps", type=int, default=5,
                    help="timed steps of the degree-120 sub-measurement (0 = skip it)")
    ap.add_argument("--e2e-depth", type=int, default=E2E_DEPTH,
                    help="batches in flight in the end-to-end leg (worker pipelines of the context)")
    ap.add_argument("--shard", action="store_true",
                    help="key-range sharding of one batch over the ranks (rfr_factor_batch_sharded; the "
                         "degree-120 workload unless --config names another) instead of replicas")
    return ap.parse_args()


def workload(cfg, rank, count):
    import workloads as W
    seeds = {"cfg1": 1, "cfg2": 2, "cfg3": 3, "cfg5": 5}
    make = {"cfg1": W.config1, "cfg2": W.config2, "cfg3": W.config3, "cfg5": W.config5}[cfg]
    insts = make(seeds[cfg] + 1000 * rank)
    return insts[:count] if count else insts


WORKLOAD_NAME = {
    "cfg1": "degree-24 product (12+12, coeffs [-10,10]) + random degree-24",
    "cfg2": "50 x degree 60, coeffs [-100,100], half products of 2-3 factors",
    "cfg3": "32 x degree 100, coeffs [-100,100], half products (50+50 or 3 factors), half random",
    "cfg5": "degree 120 = product of two random degree-60 factors, coeffs [-100,100]",
}


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


# The fused match reads its keys from L2-resident sorted lists and keeps its
# tables in shared memory: it is bound by integer instruction issue, not HBM.
# Peak: 148 SMs x 4 sub-partitions x 32 INT32 lanes x the maximum SM clock
# (2032 MHz in MEASURED_PEAKS.json), one 32-bit integer operation per lane per
# clock.  Algorithmic work: ALU_OPS_PER_HALF_SUM 32-bit operations per half-sum
# (64-bit key add 2, unit/window compare 2, fingerprint shift 1, bin or cell
# index 1, table insert or bitmap probe 2).
ALU_OPS_PER_HALF_SUM = 8


def alu_peak():
    try:
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
        kind = "derived: 148 SMs x 128 INT32 lanes x measured sm_max_mhz"
    except (OSError, KeyError, ValueError):
        mhz, kind = 2032.0, "derived: 148 SMs x 128 INT32 lanes x 2032 MHz (nominal)"
    return 148 * 128 * mhz * 1e6 / 1e9, kind      # Gop/s


KERNEL_SOURCE = {"k_join": "k_match.cu", "k_runs": "k_match.cu", "k_mitm": "k_mitm.cu"}


def profile_figure(name, key):
    """Figure `key` (per half-sum) of kernel `name` from its committed ncu
    summary (profiles/<name>_*.md: '<key>: X', 'source_sha256: H'); None if
    there is no summary or the kernel source changed since it was taken."""
    import glob
    src = os.path.join(ROOT, "paper_2410_15880_b300", "csrc", KERNEL_SOURCE[name])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{name}_*.md"))):
        txt = open(f).read()
        m = re.search(rf"{key}:\s*([0-9.eE+-]+)", txt)
        h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
        if m and h and h.group(1) == sha:
            return float(m.group(1))
    return None


def kernel_traffic(name, half_sums):
    """DRAM bytes per launch for kernel `name` from its committed ncu summary
    (dram_bytes_per_half_sum, scaled to the launch's half-sums), or None."""
    x = profile_figure(name, "dram_bytes_per_half_sum")
    return None if x is None else x * half_sums


def issue_peak():
    """Warp-instruction issue peak: 148 SMs x 4 schedulers x the measured
    maximum SM clock, one warp instruction per scheduler per clock (G/s)."""
    try:
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        mhz = 2032.0
    return 148 * 4 * mhz * 1e6 / 1e9


def serving_leg(device, n_requests, loads, max_inflight=4, max_batch=64, trace_path=""):
    """Serving stream (degrees uniform in [20,100], coefficients in [-1000,1000],
    30 % products): closed-loop capacity first (every request submitted at
    once, so batches are full), then for each load in `loads` Poisson arrivals
    at load x capacity through rfr_submit / rfr_wait; latency = completion -
    arrival on the host clock."""
    import workloads as W
    from paper_2410_15880_b300 import Context
    from paper_2410_15880_b300._native import _coeff_array
    reqs = W.config4(4, count=n_requests)
    gold = {}
    gpath = os.path.join(ROOT, "tests", "golden", "cfg4_sample.json")
    if os.path.exists(gpath):
        gold = {g["index"]: g["factors"] for g in json.load(open(gpath))}
    out = {"requests": len(reqs), "max_inflight": max_inflight, "max_batch": max_batch,
           "workload": "degrees uniform [20,100], coeffs [-1000,1000], 30% products, Poisson arrivals",
           "loads": []}
    with Context(device=device, max_inflight=max_inflight, max_batch=max_batch) as srv:
        # warm-up
        for t in [srv.submit(r.coeffs) for r in reqs[:64]]:
            srv.wait(t)
        arrs = [_coeff_array(r.coeffs) for r in reqs]          # request buffers made before timing
        t0 = time.perf_counter()
        tickets = [srv.submit(a) for a in arrs]
        for t in tickets:
            srv.wait(t)
        cap = len(reqs) / (time.perf_counter() - t0)
        out["capacity_polys_per_s"] = cap
        ok, golden_ok = True, True
        for load in loads:
            rate = load * cap
            # open loop: arrivals of the workload rescaled to `rate`
            scale = reqs[-1].arrival_s / (len(reqs) / rate)
            arrivals = [r.arrival_s / scale for r in reqs]
            done_at = [0.0] * len(reqs)
            submit_at = [0.0] * len(reqs)
            results = [None] * len(reqs)
            tick = [0] * len(reqs)
            ready = threading.Semaphore(0)

            def waiter():
                # poll every outstanding ticket (one rfr_poll_batch call per sweep), so that
                # each request is timed at its own completion: waiting on the tickets in
                # order would time a fast request only after the slower ones before it
                pending, nxt = [], 0
                while nxt < len(reqs) or pending:
                    if not pending and nxt < len(reqs):
                        ready.acquire()
                        pending.append(nxt)
                        nxt += 1
                    while nxt < len(reqs) and ready.acquire(blocking=False):
                        pending.append(nxt)
                        nxt += 1
                    got = srv.poll_batch([tick[i] for i in pending])
                    now = time.perf_counter()
                    still = []
                    for i, r in zip(pending, got):
                        if r is None:
                            still.append(i)
                        else:
                            results[i], done_at[i] = r, now
                    pending = still
                    if pending:
                        time.sleep(0.0003)

            th = threading.Thread(target=waiter)
            gc.collect()
            gc.disable()                          # no collector pauses on the client side while timing
            th.start()
            start = time.perf_counter()
            for i in range(len(reqs)):
                now = time.perf_counter() - start
                if arrivals[i] > now:
                    time.sleep(arrivals[i] - now)
                submit_at[i] = time.perf_counter()
                tick[i] = srv.submit(arrs[i])
                ready.release()
            th.join()
            gc.enable()
            if trace_path:
                with open(f"{trace_path}.load{load}.csv", "w") as fh:
                    fh.write("arrival_ms,submit_ms,done_ms,degree\n")
                    for i, r in enumerate(reqs):
                        fh.write(f"{arrivals[i] * 1e3:.3f},{(submit_at[i] - start) * 1e3:.3f},"
                                 f"{(done_at[i] - start) * 1e3:.3f},{len(r.coeffs) - 1}\n")
            makespan = max(done_at) - start
            lat = sorted((done_at[i] - start - arrivals[i]) * 1e3 for i in range(len(reqs)))
            srv_lat = sorted((done_at[i] - submit_at[i]) * 1e3 for i in range(len(reqs)))
            q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
            qs = lambda f: srv_lat[min(len(srv_lat) - 1, int(f * len(srv_lat)))]
            ok = ok and all(x is not None and x.ok for x in results)
            golden_ok = golden_ok and all(results[i].factors == f for i, f in gold.items() if i < len(results))
            out["loads"].append({"load": load, "rate_per_s": rate, "p50_ms": q(0.50), "p99_ms": q(0.99),
                                 "max_ms": lat[-1], "throughput_polys_per_s": len(reqs) / makespan,
                                 "from_submit_p50_ms": qs(0.50), "from_submit_p99_ms": qs(0.99)})
    out["all_ok"] = ok
    out["golden_checked"] = sum(1 for i in gold if i < len(reqs))
    out["golden_ok"] = golden_ok
    return out


def cpu_oracle_sample(insts, budget_s=15.0, max_polys=8):
    from oracle import factor as oracle_factor
    t0 = time.perf_counter()
    done = 0
    for inst in insts[:max_polys]:
        oracle_factor(inst.coeffs, construction=inst.factors)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done, dt


def cpu_mt_sample(d_co, d_dg, root_mode, budget_s=15.0, max_polys=8):
    """The multithreaded CPU Horowitz-Sahni band join (baseline/hs_mt.cpp) on
    the match stage of the first polynomials of the workload, over all host
    cores.  Its inputs (weights, windows, half split) come from the GPU
    path's roots and weights stages; the first polynomial is run once untimed
    to allocate and first-touch the buffers."""
    import baseline
    from paper_2410_15880_b300 import PLAN_DTYPE, stage_roots, stage_weights
    roots, radius, status = stage_roots(d_co, d_dg, root_mode)
    plans = stage_weights(d_co, d_dg, roots, radius, status).cpu().numpy().view(PLAN_DTYPE).reshape(-1)
    plans = [p for p in plans if p["status"] == 0 and int(p["window"]) < (1 << 63)]
    cores = baseline.host_cores()

    def run(p):
        na, nb = int(p["n_a"]), int(p["n_b"])
        w, w2 = [int(x) for x in p["w"]], [int(x) for x in p["w2"]]
        _, counts, _ = baseline.hs_mt_match(w[:na], w2[:na], w[na:na + nb], w2[na:na + nb],
                                            int(p["window"]), int(p["window2"]), threads=cores)
        return (1 << na) + (1 << nb), counts[1]

    if not plans:
        return None
    run(plans[0])
    done, hs, cands, t0 = 0, 0, 0, time.perf_counter()
    for p in plans[:max_polys]:
        h, c = run(p)
        done, hs, cands = done + 1, hs + h, cands + c
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "horowitz-sahni-mt",
            "half_sums_per_s": hs / dt, "candidates": cands,
            "sample": f"match stage only (sorted low lists by merging, runs, key units with a binned half a and "
                      f"an occupancy bitmap, Tr2 test; C++ std::thread) of the first {done} polynomials ({dt:.1f} s), "
                      f"weights from the GPU path's weights stage"}


def degree120_leg(ctx, flush, steps, warmup=2):
    """The degree-120 workload (one product of two random degree-60 factors,
    halves of about 2^31 + 2^32 half-sums) through the same context, timed the
    same way as the headline (device-resident input, L2 flush before each
    step, CUDA events), checked against its golden factor list."""
    import numpy as np
    import torch
    inst = workload("cfg5", 0, 0)[0]
    arr = np.zeros((1, 129), dtype=np.int64)
    arr[0, :len(inst.coeffs)] = inst.coeffs
    d_co = torch.from_numpy(arr).cuda()
    d_dg = torch.tensor([inst.degree], dtype=torch.int32, device="cuda")
    for i in range(warmup):
        ctx.factor_batch_device(d_co, d_dg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    diags = []
    e0.record()
    for i in range(steps):
        flush.fill_(i & 255)
        torch.cuda.current_stream().synchronize()
        res = ctx.factor_batch_device(d_co, d_dg)
        diags.append(res[0].diag)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    d = diags[-1]
    gpath = os.path.join(ROOT, "tests", "golden", "cfg5.json")
    gold = json.load(open(gpath))[0]["factors"] if os.path.exists(gpath) else None
    return {"workload": WORKLOAD_NAME["cfg5"], "steps": steps, "ms_per_poly": ms, "polys_per_s": 1e3 / ms,
            "n": d["n"], "n_a": d["n_a"], "n_b": d["n_b"], "half_sums": d["half_sums"],
            "half_sums_per_s": d["half_sums"] / (ms / 1e3),
            "match_ms": statistics.mean(x["stage_us"][4] for x in diags) / 1e3,
            "lists_ms": statistics.mean(x["stage_us"][2] for x in diags) / 1e3,
            "matches_golden": (gold is not None and res[0].ok and res[0].factors == gold)}


def degree60_leg(ctx, flush, steps, depth, warmup=5):
    """The degree-60 workload (50 polynomials, halves of about 2^15 + 2^16
    half-sums) through the same context: device-resident blocking calls timed
    like the headline, and end to end from pinned host rows with `depth`
    asynchronous batches in flight; both checked against the goldens."""
    import numpy as np
    import torch
    insts = workload("cfg2", 0, 0)
    arr = np.zeros((len(insts), 129), dtype=np.int64)
    for i, inst in enumerate(insts):
        arr[i, :len(inst.coeffs)] = inst.coeffs
    d_co = torch.from_numpy(arr).cuda()
    d_dg = torch.tensor([inst.degree for inst in insts], dtype=torch.int32, device="cuda")
    h_co = torch.from_numpy(arr).pin_memory().numpy()
    h_dg = np.array([inst.degree for inst in insts], dtype=np.int32)
    gpath = os.path.join(ROOT, "tests", "golden", "cfg2.json")
    gold = [g["factors"] for g in json.load(open(gpath))] if os.path.exists(gpath) else None
    for i in range(warmup):
        ctx.factor_batch_device(d_co, d_dg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(steps):
        flush.fill_(i & 255)
        torch.cuda.current_stream().synchronize()
        res = ctx.factor_batch_device(d_co, d_dg)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    d = res[0].diag

    def pipelined(n):
        pend, last = [], None
        for i in range(n):
            flush.fill_(i & 255)
            torch.cuda.current_stream().synchronize()
            pend.append(ctx.factor_batch_async(h_co, h_dg))
            if len(pend) == depth or i == n - 1:
                while pend and (len(pend) == depth or i == n - 1):
                    last = pend.pop(0).result()
        return last

    pipelined(max(3, warmup))
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    r2 = pipelined(steps)
    t1.record()
    torch.cuda.synchronize()
    ms_e2e = t0.elapsed_time(t1) / steps
    ok = gold is not None and all(r.ok and r.factors == g for r, g in zip(res, gold)) and \
        all(r.ok and r.factors == g for r, g in zip(r2, gold))
    return {"workload": WORKLOAD_NAME["cfg2"], "steps": steps, "polys_per_step": len(insts),
            "polys_per_s": len(insts) * 1e3 / ms, "ms_per_step": ms,
            "e2e": {"polys_per_s": len(insts) * 1e3 / ms_e2e, "ms_per_step": ms_e2e,
                    "api": f"rfr_factor_batch_async + rfr_batch_wait, {depth} batches in flight"},
            "roots_ms": d["stage_us"][0] / 1e3, "match_ms": d["stage_us"][4] / 1e3,
            "graphs_per_step": d["graphs"], "matches_golden": ok}


def tuned_summary(path):
    """The layouts the autotuner picked during warm-up, from its cache file:
    per (n_a, n_b) class the fused match's key-unit size and bin limit (or the
    table match's low-list bits, bucket digit and CTAs per SM)."""
    picked = {}
    try:
        for line in open(path):
            f = line.rstrip("\n").split("\t")[-1].split()
            if len(f) == 7:
                na, nb, lmax, d1o, cps, ulog, nbl = map(int, f)
                picked[f"{na}+{nb}"] = {"unit_keys_log2": ulog, "bins_log2_max": nbl, "table_l_max": lmax,
                                       "table_d1_off": d1o, "table_cta_per_sm": cps}
    except OSError:
        pass
    return {"on": True, "knobs": "fused match: key-unit size 2^12..2^14 half-a keys, bins per unit "
                                 "2^12..2^13; table match: low-list bits, bucket digit, CTAs per SM; "
                                 "timed per (n_a, n_b) class during warm-up", "picked": picked}


def sharded_leg(ctx, polys, rank, world, steps, warmup, gather, golden=None, sync=None, barrier=None):
    """Key-range shard `rank` of `world` of one batch: every rank factors the
    same polynomials, its fused matches searching only its share of the key
    units, and the verified divisor sets of all shards meet through `gather`
    before the atoms, so every rank returns the whole factorisation.  The
    steps are bracketed by `sync` (the device) and `barrier` (the ranks); the
    time is the max over ranks.  Returns (ms per step, last results, every
    result equal to `golden`)."""
    sync = sync or (lambda: None)
    barrier = barrier or (lambda: None)
    for _ in range(warmup):
        ctx.factor_batch_sharded(polys, rank, world, gather)
    sync()
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        res = ctx.factor_batch_sharded(polys, rank, world, gather)
    sync()
    barrier()
    ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / steps, world)
    ok = golden is not None and all(r.ok and r.factors == g for r, g in zip(res, golden))
    return ms, res, ok


def run_sharded(a):
    """`--shard`: one batch split by key range over the ranks (strong scaling),
    the exchange through torch.distributed's all-gather, checked on every rank
    against the golden factor lists."""
    import torch
    import torch.distributed as dist
    from paper_2410_15880_b300 import Context
    from paper_2410_15880_b300.sharding import torch_gather
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    cfg = a.config if a.config != "cfg3" else "cfg5"
    insts = workload(cfg, 0, a.count)                       # the same batch on every rank
    polys = [inst.coeffs for inst in insts]
    gpath = os.path.join(ROOT, "tests", "golden", f"{cfg}.json")
    golden = [g["factors"] for g in json.load(open(gpath))][:len(polys)] if os.path.exists(gpath) else None
    gather = torch_gather() if world > 1 else None                 # one shard: no exchange
    with Context(device=local) as ctx:
        ms, res, ok = sharded_leg(ctx, polys, rank, world, a.steps, a.warmup, gather, golden,
                                  sync=torch.cuda.synchronize, barrier=(dist.barrier if world > 1 else None))
    oks = [ok]
    if world > 1:
        oks = [None] * world
        dist.all_gather_object(oks, ok)
    if rank == 0:
        half_sums = sum(r.diag["half_sums"] for r in res)
        print(json.dumps({
            "metric": f"polynomials factored/sec, one batch key-range sharded over {world} GPU(s)",
            "value": len(polys) / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "int64+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME[cfg], "polys_per_step": len(polys), "half_sums_per_step": half_sums,
                       "parallelism": f"key-range shards x{world}", "exchange": "torch.distributed all_gather_object"},
            "half_sums_per_s": half_sums / (ms / 1e3),
            "correct": {"matches_golden_every_rank": all(oks)}}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def max_over_ranks(value: float, world: int) -> float:
    """Max of a per-rank time over all ranks (the slowest replica sets the
    step time).  Uses a CUDA tensor under NCCL, a CPU tensor under gloo."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(a):
    """The oracle as it stands, timed on host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    insts = workload(a.config, 0, a.count)
    for i in range(a.warmup):
        cpu_oracle_sample(insts[i % len(insts):], budget_s=0.0, max_polys=1)
    t0 = time.perf_counter()
    n = 0
    for i in range(a.steps):
        d, _ = cpu_oracle_sample(insts[(i % len(insts)):], budget_s=0.0, max_polys=1)
        n += d
    dt = time.perf_counter() - t0
    v = n / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * dt / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME[a.config], "sample": "one polynomial per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{n} polynomials of the workload, one per step (CPU oracle: roots, Sturm, DDF irreducibility certificates)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.shard:
        return run_sharded(a)
    import numpy as np
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2410_15880_b300 import Context
    insts = workload(a.config, rank, a.count)
    B = len(insts)
    arr = np.zeros((B, 129), dtype=np.int64)
    for i, inst in enumerate(insts):
        arr[i, :len(inst.coeffs)] = inst.coeffs
    d_co = torch.from_numpy(arr).cuda()
    d_dg = torch.tensor([inst.degree for inst in insts], dtype=torch.int32, device="cuda")
    polys = [inst.coeffs for inst in insts]
    # the end-to-end legs' inputs: the same rows in pinned host memory
    h_co = torch.from_numpy(arr).pin_memory().numpy()
    h_dg = np.array([inst.degree for inst in insts], dtype=np.int32)

    def barrier():
        if world > 1:
            dist.barrier()

    flush = torch.empty((256 << 20,), dtype=torch.uint8, device="cuda")     # larger than L2 (126 MB)
    match_path = {"auto": 0, "tables": 1, "splat": 2, "prune": 3}[a.match_path]
    # the tuned layouts are read back from the cache file (a fresh one unless --tune-cache names one)
    tune_cache = a.tune_cache
    if not tune_cache and not a.no_autotune:
        import tempfile
        tune_cache = os.path.join(tempfile.mkdtemp(prefix="rfr_tune_"), "tune.txt")
    with Context(device=local, timing=True, root_mode=a.root_mode, autotune=not a.no_autotune,
                 tune_cache_path=tune_cache, match_path=match_path, max_inflight=max(1, a.e2e_depth),
                 use_graphs=not a.no_graphs) as ctx:
        for i in range(a.warmup):
            flush.fill_(i & 255)                   # the flush kernel's first use loads it (not timed)
            torch.cuda.current_stream().synchronize()
            res = ctx.factor_batch_device(d_co, d_dg)
        # objects made before the timed regions (imports, workloads, warm-up) move to
        # the collector's permanent generation: its collections during the timed
        # calls then scan only what those calls create
        gc.collect()
        gc.freeze()
        # ---- timed region: device-resident inputs
        clocks = Clocks(local)
        clocks.start()
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        per_step = []
        for i in range(a.steps):
            flush.fill_(i & 255)
            torch.cuda.current_stream().synchronize()
            res = ctx.factor_batch_device(d_co, d_dg)
            per_step.append(res[0].diag)
        ev1.record()
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        ms = max_over_ranks(ev0.elapsed_time(ev1), world)
        statuses = [r.status for r in res]
        # ---- correctness of the last timed step (outside the timed region)
        ok_golden = None
        gpath = os.path.join(ROOT, "tests", "golden", f"{a.config}.json")
        if rank == 0 and os.path.exists(gpath):
            gold = json.load(open(gpath))[:B]
            ok_golden = all(r.ok and r.factors == g["factors"] for r, g in zip(res, gold))
        # ---- e2e: host buffers through rfr_factor_batch_async, `depth` batches
        # in flight, one per worker pipeline (each on its own stream): while
        # they run, this thread queues the next batch and turns the oldest
        # finished one's results into Python objects
        depth = max(1, a.e2e_depth)

        def e2e_pipelined(steps, lat, stages):
            pend, last = [], None
            for i in range(steps):
                flush.fill_(i & 255)
                torch.cuda.current_stream().synchronize()
                pend.append((ctx.factor_batch_async(h_co, h_dg), time.perf_counter()))
                if len(pend) == depth or i == steps - 1:
                    while pend and (len(pend) == depth or i == steps - 1):
                        h, t0 = pend.pop(0)
                        last = h.result()
                        lat.append((time.perf_counter() - t0) * 1e3)
                        stages.append(last[0].diag["stage_us"])
            return last

        e2e_pipelined(max(3, a.warmup), [], [])
        for _ in range(max(2, a.warmup)):
            ctx.factor_batch(h_co, h_dg)
        gc.collect()
        gc.freeze()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        e2e_lat, e2e_stage = [], []
        r2 = e2e_pipelined(a.steps, e2e_lat, e2e_stage)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1), world)
        e2e_diag = r2[0].diag
        # the same through the blocking rfr_factor_batch, one batch at a time
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        sync_stage, sync_wall = [], []
        for i in range(a.steps):
            flush.fill_(i & 255)
            torch.cuda.current_stream().synchronize()
            t0 = time.perf_counter()
            rs = ctx.factor_batch(h_co, h_dg)
            sync_wall.append((time.perf_counter() - t0) * 1e3)
            sync_stage.append(rs[0].diag["stage_us"])
        s1.record()
        torch.cuda.synchronize()
        barrier()
        ms_sync = max_over_ranks(s0.elapsed_time(s1), world)
        # ---- the degree-120 workload (rank 0, default headline workload only)
        deg120 = None
        if rank == 0 and world == 1 and a.config == "cfg3" and a.degree120_steps > 0:
            deg120 = degree120_leg(ctx, flush, a.degree120_steps)
        # ---- the degree-60 workload (rank 0, default headline workload only)
        deg60 = None
        if rank == 0 and world == 1 and a.config == "cfg3" and a.degree60_steps > 0:
            deg60 = degree60_leg(ctx, flush, a.degree60_steps, depth)
        # ---- one launch per polynomial (same inputs, host buffers)
        one_ms = None
        if rank == 0:
            torch.cuda.synchronize()
            o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            o0.record()
            singles = [ctx.factor(p) for p in polys]
            o1.record()
            torch.cuda.synchronize()
            one_ms = o0.elapsed_time(o1)
            single_ok = [s.factors for s in singles] == [r.factors for r in r2]

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    half_sums = sum(r.diag["half_sums"] for r in res)
    polys_total = B * world * a.steps
    value = polys_total / (ms / 1e3)
    # dominant kernel: average launch durations from the library's CUDA events
    join_us = statistics.mean(d["stage_us"][4] for d in per_step)
    scat_us = statistics.mean(d["stage_us"][3] for d in per_step)
    count_us = statistics.mean(d["stage_us"][2] for d in per_step)
    roots_us = statistics.mean(d["stage_us"][0] for d in per_step)
    peak, peak_kind = peaks()
    fused = all(d["stage_us"][3] < 0.05 * d["stage_us"][4] for d in per_step)
    if a.match_path == "splat":
        # splat match: fill 2 cells (16 B) and one exchange (8 B read + 8 B write) per
        # half-b sum, one 8 B cell read per half-a sum, at the least
        alg_bytes = sum(32.0 * (1 << r.diag["n_b"]) + 8.0 * (1 << r.diag["n_a"]) for r in res)
        achieved = alg_bytes / (join_us * 1e-6) / 1e9
        roof = {"bound": "hbm", "kernel": "k_splat_insert+k_splat_query", "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "algorithmic_bytes": alg_bytes, "avg_launch_us": join_us}
    elif a.match_path == "prune":
        # Algorithm B: integer ALU work per visited pattern (acceptance test, trailing
        # zeros, jump search, O(1) value update), about 20 operations
        apeak, apeak_kind = alu_peak()
        visited = sum(r.diag["cand_coarse"] for r in res)
        ops = 20.0 * visited
        achieved = ops / (join_us * 1e-6) / 1e9
        roof = {"bound": "alu", "kernel": "k_prune", "achieved": achieved, "peak": apeak,
                "peak_kind": apeak_kind, "unit": "Gop/s", "frac": achieved / apeak, "traffic": None,
                "algorithmic_ops": ops, "patterns_visited": visited, "avg_launch_us": join_us}
    elif fused:
        # the fused match (k_mitm) is the match stage; no table scatter ran.  Three
        # fractions: integer operations against the INT32 peak (the primary line),
        # the method's HBM floor (each half written once and read once, 24 B per
        # half-sum) against the measured HBM peak, and the warp instructions the
        # committed ncu summary counts per half-sum against the issue peak.
        apeak, apeak_kind = alu_peak()
        ops = ALU_OPS_PER_HALF_SUM * half_sums
        achieved = ops / (join_us * 1e-6) / 1e9
        hbm_eq = 24.0 * half_sums / (join_us * 1e-6) / 1e9
        ipk = issue_peak()
        inst = profile_figure("k_mitm", "warp_inst_per_half_sum")
        issue = None if inst is None else inst * half_sums / (join_us * 1e-6) / 1e9
        roof = {"bound": "alu", "kernel": "k_mitm", "achieved": achieved, "peak": apeak,
                "peak_kind": apeak_kind, "unit": "Gop/s", "frac": achieved / apeak,
                "traffic": kernel_traffic("k_mitm", half_sums),
                "algorithmic_ops": ops, "avg_launch_us": join_us,
                "hbm_equivalent": {"bytes_per_half_sum": 24, "achieved_GBps": hbm_eq, "peak_GBps": peak,
                                   "peak_kind": peak_kind, "frac": hbm_eq / peak},
                "issue": {"warp_inst_per_half_sum": inst, "achieved_Ginst_per_s": issue, "peak_Ginst_per_s": ipk,
                          "peak_kind": "148 SMs x 4 schedulers x measured sm_max_mhz",
                          "frac": None if issue is None else issue / ipk,
                          "source": "profiles/k_mitm_deg100.md (null if the kernel changed since)"}}
    else:
        kern = {"k_join": (join_us, 8.0 * half_sums), "k_runs": (scat_us, 8.0 * half_sums)}
        dom = max(kern, key=lambda k: kern[k][0])
        dur_us, alg_bytes = kern[dom]
        achieved = alg_bytes / (dur_us * 1e-6) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": kernel_traffic(dom, half_sums),
                "algorithmic_bytes": alg_bytes, "avg_launch_us": dur_us}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME[a.config], "polys_per_step": B,
                   "half_sums_per_step": half_sums, "parallelism": f"replicas x{world}",
                   "l2": "256 MiB buffer written before every timed step (L2 flush)", "root_mode": a.root_mode,
                   "autotune": "off" if a.no_autotune else tuned_summary(tune_cache),
                   "graphs": ("off" if a.no_graphs else
                              f"on: {per_step[-1]['graphs']} replayed per device-resident step "
                              "(the fused match's launch sequence; host inputs add the prologue)"),
                   "match_path": a.match_path},
        "half_sums_per_s": half_sums * world * a.steps / (ms / 1e3),
        # what a design that keeps the sorted halves in HBM would need to move for the same
        # half-sums/s: 128 B per half-sum for enumerate + 4 LSD passes + join, 24 B at the
        # method's floor (each table written once and read once)
        "hbm_model": {"bytes_per_half_sum_sorted_tables": 128, "bytes_per_half_sum_floor": 24,
                      "equivalent_GBps_sorted_tables": 128 * half_sums * a.steps / (ms / 1e3) / 1e9,
                      "equivalent_GBps_floor": 24 * half_sums * a.steps / (ms / 1e3) / 1e9,
                      "hbm_peak_GBps": peak},
        "roofline": roof,
        "stage_us_per_step": {"validate+roots": roots_us,
                              "weights": statistics.mean(d["stage_us"][1] for d in per_step),
                              "lists+count+scans": count_us, "scatter": scat_us, "match": join_us,
                              "verify+atoms": statistics.mean(d["stage_us"][5] for d in per_step),
                              "host_total": statistics.mean(d["stage_us"][7] for d in per_step),
                              "device_total": statistics.mean(d["stage_us"][6] for d in per_step)},
        "e2e": {"value": polys_total / (ms_e2e / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(e2e_diag["h2d_bytes"]), "d2h_bytes_per_step": int(e2e_diag["d2h_bytes"]),
                "ms_per_step": ms_e2e / a.steps,
                "api": f"rfr_factor_batch_async + rfr_batch_wait, {depth} batches in flight (L2 flush before each submit); "
                       "inputs: int64 rows in pinned host memory",
                "batch_latency_ms_median": statistics.median(e2e_lat), "batch_latency_ms_max": max(e2e_lat),
                "library_host_us_per_step": statistics.mean(x[7] for x in e2e_stage),
                "library_device_us_per_step": statistics.mean(x[6] for x in e2e_stage),
                "blocking_call": {"value": polys_total / (ms_sync / 1e3), "unit": UNIT,
                                  "api": "rfr_factor_batch, one batch at a time",
                                  "ms_per_step": ms_sync / a.steps,
                                  "call_ms_median": statistics.median(sync_wall), "call_ms_max": max(sync_wall),
                                  "library_host_us_per_step": statistics.mean(x[7] for x in sync_stage)}},
        "one_launch_per_polynomial": {"value": B / (one_ms / 1e3), "unit": UNIT, "same_factors": single_ok},
        "gpu_launches": int(sum(d["launches"] for d in per_step)),
        "clocks": clk,
        "correct": {"statuses_ok": all(s == 0 for s in statuses), "matches_golden": ok_golden},
    }
    if deg120 is not None:
        line["degree120"] = deg120
    if deg60 is not None:
        line["degree60"] = deg60
    if a.serving_requests > 0 and world == 1:
        line["serving"] = serving_leg(local, a.serving_requests, [float(x) for x in a.serving_loads.split(",")],
                                      trace_path=a.serving_trace)
    if not a.no_cpu_baseline and world == 1:         # the CPU baselines run at N = 1 only
        n, dt = cpu_oracle_sample(workload(a.config, 0, a.count), budget_s=15.0)
        line["cpu_baseline"] = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {n} polynomials of the workload ({dt:.1f} s): roots, Sturm, DDF certificates"}
        mt = cpu_mt_sample(d_co, d_dg, a.root_mode)
        if mt is not None:
            line["cpu_mt"] = mt
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
