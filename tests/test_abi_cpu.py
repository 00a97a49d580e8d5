"""C-ABI checks that need no GPU: the library builds, loads, exports every
function the headers declare, and its host-only entry points behave."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in ("rfr.h", "rfr_stages.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(rfr_[a-z_0-9]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def L():
    from paper_2410_15880_b300.build import build
    build()
    import paper_2410_15880_b300 as P
    return P.lib()


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n


def test_host_only_calls(L):
    import paper_2410_15880_b300._native as N
    assert L.rfr_version().startswith(b"rfr-b300")
    assert L.rfr_strerror(-8) == b"too many candidate patterns"
    assert L.rfr_strerror(12345) == b"unknown status"
    cfg = N.Config()
    assert L.rfr_config_default(ctypes.byref(cfg)) == 0
    assert cfg.max_inflight == 2 and cfg.max_candidates == 1 << 16 and cfg.root_mode == 1
    assert cfg.use_graphs == 1 and cfg.autotune == 0 and not cfg.tune_cache_path
    assert cfg.match_path == 0
    assert L.rfr_config_default(None) == -1
    assert L.rfr_destroy(None) == 0
    f = N.Factors()
    L.rfr_factors_free(ctypes.byref(f))                 # zeroed struct is fine


def test_struct_layout(L):
    import paper_2410_15880_b300._native as N
    assert N.PLAN_DTYPE.itemsize == 2512
    assert ctypes.sizeof(N.Config) == 72 and ctypes.sizeof(N.Diag) == 184


def test_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2410_15880_b300._native as N
    h = ctypes.c_void_p()
    assert L.rfr_create(None, ctypes.byref(h)) == -13     # RFR_E_CUDA, no abort
    assert not h.value


def test_stage_argument_checks(L):
    # invalid sizes are rejected on the host before any launch
    assert L.rfr_stage_enumerate(None, 4, None, None) == -1
    assert L.rfr_stage_match_workspace(5, 3) == 0          # n_b < n_a is not a valid split
    assert L.rfr_stage_match_workspace(10, 11) > (1 << 11) * 8
    assert L.rfr_stage_match_fused_workspace(1, 2) == 0    # the fused match needs two elements per half
    assert L.rfr_stage_match_fused_workspace(12, 33) == 0  # and at most 32
    assert L.rfr_stage_match_fused_workspace(26, 27) > (1 << 20) * (8 + 4 + 4 + 4)   # lists, masks, directory, positions
    # the host-side bound check of the fused geometry (k_mitm indexes its table
    # and bitmap without clamps) accepts every pair of half sizes it takes
    assert all(L.rfr_stage_match_fused_workspace(a, b) > 0 for a in range(2, 33) for b in range(a, 33))
    assert L.rfr_stage_splat_cells(-1) == 0 and L.rfr_stage_splat_cells(31) == 0
    assert L.rfr_stage_splat_cells(10) == (2 << 10) + 4096 + 32   # home cells, overflow cells, descriptor
    assert L.rfr_stage_splat(None, 40, None, 0, None, None) == -1


def test_golden_files_are_consistent():
    from oracle.zpoly import pmul
    for name in ("cfg1", "cfg2", "cfg3", "cfg4_sample", "cfg5", "special"):
        recs = json.load(open(os.path.join(ROOT, "tests", "golden", f"{name}.json")))
        for r in recs:
            assert "factors" in r, r["name"]
            acc = [1]
            for f in r["factors"]:
                assert f[-1] == 1
                acc = pmul(acc, f)
            assert acc == r["coeffs"], r["name"]


def test_batch_results_flattened_and_released(L):
    """A batch's results as the library hands them over (malloc'ed arrays per
    result) become factor lists through one rfr_factors_flatten copy; every
    array is released, error results carry no factors, and the diagnostics are
    read from the result array itself."""
    import paper_2410_15880_b300._native as N
    libc = ctypes.CDLL(None)
    libc.malloc.restype = ctypes.c_void_p
    libc.malloc.argtypes = [ctypes.c_size_t]
    facs = [[[-7, 1], [1, 0, 1], [3, 2, 1]], None, [[5, 0, 0, 1]], []]
    n = len(facs)
    outs = (N.Factors * n)()
    sts = (ctypes.c_int * n)(0, -5, 0, 0)
    for i, fs in enumerate(facs):
        outs[i].diag.n = 10 + i
        if not fs:
            continue
        co = [c for f in fs for c in f]
        d = libc.malloc(4 * len(fs))
        c = libc.malloc(8 * len(co))
        (ctypes.c_int * len(fs)).from_address(d)[:] = [len(f) - 1 for f in fs]
        (ctypes.c_int64 * len(co)).from_address(c)[:] = co
        outs[i].n_factors = len(fs)
        outs[i].degrees = ctypes.cast(d, type(outs[i].degrees))
        outs[i].coeffs = ctypes.cast(c, type(outs[i].coeffs))
    res = N._to_results(n, sts, outs)
    assert [r.factors for r in res] == [facs[0], [], facs[2], []]
    assert [r.status for r in res] == [0, -5, 0, 0]
    assert [r.diag["n"] for r in res] == [10, 11, 12, 13]
    assert all(outs[i].n_factors == 0 and not outs[i].coeffs for i in range(n))
    # too little room: an error, nothing written past the caps
    one = (N.Factors * 1)()
    d, c = libc.malloc(4), libc.malloc(16)
    (ctypes.c_int * 1).from_address(d)[0] = 1
    (ctypes.c_int64 * 2).from_address(c)[:] = [3, 1]
    one[0].n_factors, one[0].degrees, one[0].coeffs = 1, ctypes.cast(d, type(one[0].degrees)), ctypes.cast(c, type(one[0].coeffs))
    co, dg, nf = (ctypes.c_int64 * 1)(), (ctypes.c_int32 * 1)(), (ctypes.c_int32 * 1)()
    assert L.rfr_factors_flatten(one, 1, co, 1, dg, 1, nf) == -3
    assert L.rfr_factors_flatten(one, 1, (ctypes.c_int64 * 2)(), 2, dg, 1, nf) == 2
    assert L.rfr_factors_flatten(None, 1, co, 1, dg, 1, nf) == -1
    L.rfr_factors_free_n(one, 1)
