"""ctypes declarations of the C ABI and small marshalling helpers."""
from __future__ import annotations

import ctypes as C
import itertools
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "librfr.so")

RFR_MAX_DEGREE = 128
RFR_LDC = RFR_MAX_DEGREE + 1
RFR_OK = 0
RFR_PENDING = 1
RFR_E_TIMEOUT = -12
RFR_ROOTS_FP64 = 0
RFR_ROOTS_FP32_BULK = 1
RFR_MATCH_AUTO = 0
RFR_MATCH_TABLES = 1
RFR_MATCH_SPLAT = 2
RFR_MATCH_PRUNE = 3

_STATUS = {
    0: "RFR_OK", 1: "RFR_PENDING", -1: "RFR_E_INVALID", -2: "RFR_E_NOT_MONIC",
    -3: "RFR_E_RANGE", -4: "RFR_E_NOT_SQUAREFREE", -5: "RFR_E_NO_CONVERGENCE",
    -6: "RFR_E_ROOTS", -7: "RFR_E_WINDOW", -8: "RFR_E_CAND_OVERFLOW",
    -9: "RFR_E_OVERFLOW", -10: "RFR_E_OOM", -11: "RFR_E_BUDGET", -12: "RFR_E_TIMEOUT",
    -13: "RFR_E_CUDA", -14: "RFR_E_CANCELLED", -15: "RFR_E_INTERNAL",
}


def status_name(st: int) -> str:
    return _STATUS.get(int(st), f"status {st}")


class RFRError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {status_name(status)}" if what else status_name(status))


class Config(C.Structure):
    _fields_ = [("device", C.c_int), ("mem_budget_bytes", C.c_size_t), ("max_inflight", C.c_int),
                ("max_batch", C.c_int), ("root_mode", C.c_int), ("timing", C.c_int),
                ("max_candidates", C.c_uint64), ("eps_override", C.c_double),
                ("use_graphs", C.c_int), ("autotune", C.c_int), ("tune_cache_path", C.c_char_p),
                ("match_path", C.c_int), ("reserved0", C.c_int)]


class Diag(C.Structure):
    _fields_ = [("n", C.c_int), ("r", C.c_int), ("c", C.c_int), ("n_a", C.c_int), ("n_b", C.c_int),
                ("window", C.c_uint64), ("half_sums", C.c_uint64), ("cand_coarse", C.c_uint64),
                ("cand_pre", C.c_uint64), ("cand_post", C.c_uint64), ("verified", C.c_uint64),
                ("max_rel_residual", C.c_double), ("max_root_err", C.c_double),
                ("stage_us", C.c_double * 8), ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64),
                ("launches", C.c_uint32), ("batch_size", C.c_uint32), ("graphs", C.c_uint32),
                ("reserved", C.c_uint32)]


class Factorization(C.Structure):
    _fields_ = [("content", C.c_int64), ("n_factors", C.c_int), ("degrees", C.POINTER(C.c_int)),
                ("multiplicities", C.POINTER(C.c_int)), ("coeffs", C.POINTER(C.c_int64))]


class Factors(C.Structure):
    _fields_ = [("n_factors", C.c_int), ("degrees", C.POINTER(C.c_int)),
                ("coeffs", C.POINTER(C.c_int64)), ("diag", Diag)]


# rfr_plan as a numpy structured dtype (byte-exact with include/rfr_stages.h)
PLAN_DTYPE = np.dtype([
    ("status", "<i4"), ("degree", "<i4"), ("n", "<i4"), ("r", "<i4"), ("c", "<i4"),
    ("n_a", "<i4"), ("n_b", "<i4"), ("pad0", "<i4"), ("window", "<u8"), ("window2", "<u8"),
    ("max_radius", "<f8"), ("max_rel_residual", "<f8"), ("sum_err1", "<f8"), ("sum_err2", "<f8"),
    ("w", "<u8", (RFR_MAX_DEGREE,)), ("w2", "<u8", (RFR_MAX_DEGREE,)),
    ("kind", "u1", (RFR_MAX_DEGREE,)), ("root0", "u1", (RFR_MAX_DEGREE,)),
    ("root1", "u1", (RFR_MAX_DEGREE,)),
])

_lib = None
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
GATHER_FN = C.CFUNCTYPE(C.c_int, C.POINTER(C.c_uint64), C.c_size_t, C.POINTER(C.POINTER(C.c_uint64)),
                        C.POINTER(C.c_size_t), C.c_void_p)
_libc = C.CDLL(None)
_libc.malloc.restype = C.c_void_p
_libc.malloc.argtypes = [C.c_size_t]
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


def lib():
    """The loaded librfr.so.  Raises if it was not built: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"librfr.so is not built ({_LIB_PATH}); run "
                           "`python -m paper_2410_15880_b300.build`")
    L = C.CDLL(_LIB_PATH)
    vp, i32, i64p, u64 = C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.c_uint64
    sig = {
        "rfr_version": (C.c_char_p, []),
        "rfr_strerror": (C.c_char_p, [i32]),
        "rfr_config_default": (i32, [C.POINTER(Config)]),
        "rfr_create": (i32, [C.POINTER(Config), C.POINTER(vp)]),
        "rfr_destroy": (i32, [vp]),
        "rfr_set_allocator": (i32, [vp, ALLOC_FN, FREE_FN, vp]),
        "rfr_factor": (i32, [vp, i64p, i32, C.POINTER(Factors)]),
        "rfr_factor_batch": (i32, [vp, i32, C.POINTER(i64p), C.POINTER(C.c_int), C.POINTER(Factors), C.POINTER(C.c_int)]),
        "rfr_factors_free_n": (None, [C.POINTER(Factors), i32]),
        "rfr_factors_flatten": (C.c_int64, [C.POINTER(Factors), i32, vp, C.c_size_t, vp, C.c_size_t, vp]),
        "rfr_factor_batch_device": (i32, [vp, i32, vp, vp, C.POINTER(Factors), C.POINTER(C.c_int)]),
        "rfr_factor_batch_async": (i32, [vp, i32, C.POINTER(i64p), C.POINTER(C.c_int), C.POINTER(Factors),
                                         C.POINTER(C.c_int), C.POINTER(u64)]),
        "rfr_batch_wait": (i32, [vp, u64, i32]),
        "rfr_factor_batch_sharded": (i32, [vp, i32, C.POINTER(i64p), C.POINTER(C.c_int), i32, i32, GATHER_FN, vp,
                                           C.POINTER(Factors), C.POINTER(C.c_int)]),
        "rfr_stage_validate": (i32, [vp, vp, i32, vp, vp]),
        "rfr_submit": (i32, [vp, i64p, i32, C.POINTER(u64)]),
        "rfr_poll": (i32, [vp, u64, C.POINTER(Factors)]),
        "rfr_poll_batch": (i32, [vp, i32, C.POINTER(u64), C.POINTER(Factors), C.POINTER(C.c_int)]),
        "rfr_wait": (i32, [vp, u64, i32, C.POINTER(Factors)]),
        "rfr_cancel": (i32, [vp, u64]),
        "rfr_factors_free": (None, [C.POINTER(Factors)]),
        "rfr_factor_general": (i32, [vp, i64p, i32, C.POINTER(Factorization)]),
        "rfr_squarefree": (i32, [i64p, i32, C.POINTER(Factorization)]),
        "rfr_factorization_free": (None, [C.POINTER(Factorization)]),
        "rfr_stage_roots": (i32, [vp, vp, i32, i32, vp, vp, vp, vp]),
        "rfr_stage_weights": (i32, [vp, vp, i32, vp, vp, vp, C.c_double, vp, vp]),
        "rfr_stage_enumerate": (i32, [vp, i32, vp, vp]),
        "rfr_stage_match_workspace": (C.c_size_t, [i32, i32]),
        "rfr_stage_match_fused_workspace": (C.c_size_t, [i32, i32]),
        "rfr_stage_lowlist_workspace": (C.c_size_t, [i32]),
        "rfr_stage_lowlist": (i32, [vp, i32, i32, vp, vp, vp, C.c_size_t, vp]),
        "rfr_stage_prune": (i32, [vp, vp, i32, u64, u64, vp, u64, vp, vp, C.c_size_t, vp]),
        "rfr_stage_splat_cells": (C.c_size_t, [i32]),
        "rfr_stage_splat": (i32, [vp, i32, vp, C.c_size_t, vp, vp]),
        "rfr_stage_splat_match": (i32, [vp, vp, i32, vp, vp, i32, u64, u64, vp, C.c_size_t, vp, u64, vp, vp]),
        "rfr_stage_match": (i32, [vp, vp, i32, vp, vp, i32, u64, u64, vp, C.c_size_t, vp, u64, vp, vp]),
        "rfr_stage_match_noalloc": (i32, [vp, vp, i32, vp, vp, i32, u64, u64, vp, u64, vp, vp]),
        "rfr_stage_match_exact": (i32, [vp, vp, i32, vp, vp, i32, u64, u64, vp, C.c_size_t, vp, u64, vp, vp]),
        "rfr_stage_match_fused": (i32, [vp, vp, i32, vp, vp, i32, u64, u64, vp, C.c_size_t, vp, u64, vp, vp]),
        "rfr_stage_verify": (i32, [vp, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


@dataclass
class Result:
    """One factorisation: canonical factor list plus diagnostics (the diag
    dict is built from the library's record when first read)."""
    status: int
    factors: List[List[int]] = field(default_factory=list)
    _diag: object = field(default=None, repr=False)

    @property
    def ok(self) -> bool:
        return self.status == RFR_OK

    @property
    def diag(self) -> dict:
        if not isinstance(self._diag, dict):
            d = self._diag
            if isinstance(d, tuple):                     # (the batch's result array, index)
                d = d[0][d[1]].diag
            self._diag = _diag_dict(d) if d is not None else {}
        return self._diag


_DIAG_FIELDS = [k for k, _ in Diag._fields_]


def _diag_dict(d: Diag) -> dict:
    out = {k: getattr(d, k) for k in _DIAG_FIELDS}
    out["stage_us"] = list(out["stage_us"])
    return out


def _factor_lists(n: int, degrees, coeffs) -> List[List[int]]:
    """n factors stored one after the other (degrees[i] + 1 coefficients each)."""
    if n <= 0:
        return []
    degs = degrees[:n]                                   # pointer slices: lists of Python ints
    co = coeffs[:sum(degs) + n]
    out, off = [], 0
    for e in degs:
        out.append(co[off:off + e + 1])
        off += e + 1
    return out


def _to_result(status: int, f: Factors) -> Result:
    res = Result(status=int(status), _diag=Diag.from_buffer_copy(f.diag))
    if status == RFR_OK:
        res.factors = _factor_lists(f.n_factors, f.degrees, f.coeffs)
    lib().rfr_factors_free(C.byref(f))
    return res


def _to_results(n: int, sts, outs) -> List[Result]:
    """The n results of a batch call: their factors come over in one flat copy
    (rfr_factors_flatten), their arrays are released with one call, and each
    result's diagnostics are read from `outs` when first asked for."""
    L = lib()
    nf = np.empty(n, dtype=np.int32)
    co = np.empty(n * 2 * RFR_LDC, dtype=np.int64)
    dg = np.empty(n * RFR_LDC, dtype=np.int32)
    tot = L.rfr_factors_flatten(outs, n, co.ctypes.data, co.size, dg.ctypes.data, dg.size, nf.ctypes.data)
    L.rfr_factors_free_n(outs, n)
    if tot < 0:
        raise RFRError(int(tot), "rfr_factors_flatten")
    nfl = nf.tolist()
    cl, dl = co[:tot].tolist(), dg[:sum(nfl)].tolist()
    res, oc, od = [], 0, 0
    for i, st in enumerate(sts[:n]):
        r = Result(status=st, _diag=(outs, i))
        k = nfl[i]
        if k:
            fl = []
            for e in dl[od:od + k]:
                fl.append(cl[oc:oc + e + 1])
                oc += e + 1
            od += k
            r.factors = fl
        res.append(r)
    return res


def _marshal(polys, degrees=None):
    """(n, row pointers, degrees, arrays to keep alive) for a batch call: the
    rows of an int64 array in place, or a sequence of coefficient lists
    copied one after the other into one flat buffer."""
    if isinstance(polys, np.ndarray):
        arr = np.ascontiguousarray(polys, dtype=np.int64)
        n = arr.shape[0]
        degs = np.ascontiguousarray(degrees, dtype=np.int32)
        addrs = (arr.ctypes.data + np.arange(n, dtype=np.uint64) * np.uint64(arr.strides[0])).astype(np.uint64)
    else:
        n = len(polys)
        lens = np.fromiter(map(len, polys), dtype=np.int64, count=n)
        degs = (lens - 1).astype(np.int32)
        arr = np.fromiter(itertools.chain.from_iterable(polys), dtype=np.int64, count=int(lens.sum()))
        starts = np.concatenate([np.zeros(1, dtype=np.int64), np.cumsum(lens)[:-1]]).astype(np.uint64)
        addrs = (np.uint64(arr.ctypes.data) + starts[:n] * np.uint64(8)).astype(np.uint64)
    ptrs = (C.POINTER(C.c_int64) * n).from_buffer(addrs)
    degs_c = degs.ctypes.data_as(C.POINTER(C.c_int))
    return n, ptrs, degs_c, (arr, degs, addrs)


class PendingBatch:
    """A batch queued by Context.factor_batch_async.  result() waits for it
    (rfr_batch_wait) and returns what factor_batch would have; it may be
    called again and returns the same list.  The result arrays the library
    writes into are held by the context until the batch has been waited for,
    so dropping the handle early is safe: Context.close() then waits for the
    batch and releases what it produced."""

    def __init__(self, ctx, n, outs, sts, ticket):
        self._ctx, self._n, self._ticket = ctx, n, ticket
        self._res = [] if n == 0 else None

    def result(self, timeout_ms: int = -1) -> List[Result]:
        if self._res is None:
            if not self._ctx._h or self._ticket not in self._ctx._inflight:
                raise RFRError(-1, "rfr_batch_wait: the context was closed")
            rc = lib().rfr_batch_wait(self._ctx._h, self._ticket, int(timeout_ms))
            if rc == RFR_E_TIMEOUT:
                raise RFRError(rc, "rfr_batch_wait")
            outs, sts, n = self._ctx._inflight.pop(self._ticket)
            if rc != RFR_OK:
                lib().rfr_factors_free_n(outs, n)
                self._res = RFRError(rc, "rfr_factor_batch_async")
            else:
                self._res = _to_results(n, sts, outs)
        if isinstance(self._res, RFRError):
            raise self._res
        return self._res


@dataclass
class GeneralResult:
    """p = content * prod f^m over `factors` [(f, m), ...] in canonical order."""
    status: int
    content: int = 0
    factors: List[tuple] = field(default_factory=list)

    @property
    def ok(self) -> bool:
        return self.status == RFR_OK


def _to_general(status: int, f: Factorization) -> GeneralResult:
    res = GeneralResult(status=int(status))
    if status == RFR_OK:
        res.content = int(f.content)
        fs = _factor_lists(f.n_factors, f.degrees, f.coeffs)
        res.factors = [(g, int(f.multiplicities[i])) for i, g in enumerate(fs)]
    lib().rfr_factorization_free(C.byref(f))
    return res


def squarefree(coeffs: Sequence[int]) -> GeneralResult:
    """Square-free decomposition of any nonzero p in Z[x] (rfr_squarefree, host only)."""
    f = Factorization()
    st = lib().rfr_squarefree(_coeff_array(coeffs), len(coeffs) - 1, C.byref(f))
    return _to_general(st, f)


def _coeff_array(coeffs: Sequence[int]):
    return (C.c_int64 * len(coeffs))(*coeffs)


class Context:
    """A library context (rfr_create).  Thread-safe; use as a context manager."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_inflight: int = 2,
                 max_batch: int = 64, root_mode: int = RFR_ROOTS_FP32_BULK, timing: bool = False,
                 max_candidates: int = 1 << 16, eps_override: float = 0.0, use_graphs: bool = True,
                 autotune: bool = False, tune_cache_path: Optional[str] = None, tables_only: bool = False,
                 match_path: Optional[int] = None):
        L = lib()
        cfg = Config()
        L.rfr_config_default(C.byref(cfg))
        cfg.device, cfg.mem_budget_bytes, cfg.max_inflight = device, mem_budget_bytes, max_inflight
        cfg.max_batch, cfg.root_mode, cfg.timing = max_batch, root_mode, int(bool(timing))
        cfg.max_candidates, cfg.eps_override = max_candidates, eps_override
        cfg.use_graphs, cfg.autotune = int(bool(use_graphs)), int(bool(autotune))
        cfg.tune_cache_path = tune_cache_path.encode() if tune_cache_path else None
        cfg.match_path = match_path if match_path is not None else (RFR_MATCH_TABLES if tables_only else RFR_MATCH_AUTO)
        h = C.c_void_p()
        st = L.rfr_create(C.byref(cfg), C.byref(h))
        if st != RFR_OK:
            raise RFRError(st, "rfr_create")
        self._h = h
        self._keep = []
        self._inflight = {}             # ticket -> (outs, statuses, n) of batches not yet waited for

    def close(self):
        if getattr(self, "_h", None):
            lib().rfr_destroy(self._h)      # running batches finish, queued ones are dropped
            self._h = None
            for outs, _sts, n in self._inflight.values():
                lib().rfr_factors_free_n(outs, n)
            self._inflight = {}

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_allocator(self, alloc, free):
        """Route device allocations through alloc(nbytes, stream) -> address
        (0 when it cannot) and free(address, nbytes, stream) (rfr_set_allocator);
        both None restores the built-in stream-ordered pool."""
        if alloc is None and free is None:
            st = lib().rfr_set_allocator(self._h, C.cast(None, ALLOC_FN), C.cast(None, FREE_FN), None)
            self._keep = []
        else:
            fa = ALLOC_FN(lambda nbytes, user, stream: alloc(int(nbytes), stream or 0) or None)
            ff = FREE_FN(lambda ptr, nbytes, user, stream: free(ptr, int(nbytes), stream or 0))
            st = lib().rfr_set_allocator(self._h, fa, ff, None)
            if st == RFR_OK:
                self._keep = [fa, ff]
        if st != RFR_OK:
            raise RFRError(st, "rfr_set_allocator")

    def use_torch_allocator(self):
        """Route device allocations through PyTorch's caching allocator."""
        import torch
        dev = torch.cuda.current_device()
        self.set_allocator(lambda nbytes, stream: torch.cuda.caching_allocator_alloc(nbytes, dev, stream),
                           lambda ptr, nbytes, stream: torch.cuda.caching_allocator_delete(ptr))

    def factor(self, coeffs: Sequence[int]) -> Result:
        f = Factors()
        arr = _coeff_array(coeffs)
        st = lib().rfr_factor(self._h, arr, len(coeffs) - 1, C.byref(f))
        return _to_result(st, f)

    def factor_general(self, coeffs: Sequence[int]) -> GeneralResult:
        """Any nonzero p in Z[x]: content, multiplicities, irreducible factors."""
        f = Factorization()
        st = lib().rfr_factor_general(self._h, _coeff_array(coeffs), len(coeffs) - 1, C.byref(f))
        return _to_general(st, f)

    def factor_batch(self, polys, degrees=None) -> List[Result]:
        """polys: a sequence of ascending coefficient lists, or an int64 numpy
        array [n, m] whose row i holds polynomial i (then degrees[i] gives its
        degree).  The rows are passed to rfr_factor_batch in place."""
        if len(polys) == 0:
            return []
        n, ptrs, degs_c, _keep = _marshal(polys, degrees)
        outs = (Factors * n)()
        sts = (C.c_int * n)()
        rc = lib().rfr_factor_batch(self._h, n, ptrs, degs_c, outs, sts)
        if rc != RFR_OK:
            lib().rfr_factors_free_n(outs, n)
            raise RFRError(rc, "rfr_factor_batch")
        return _to_results(n, sts, outs)

    def factor_batch_async(self, polys, degrees=None) -> "PendingBatch":
        """Queue a batch (rfr_factor_batch_async) and return at once; the
        handle's result() waits for it.  Inputs as for factor_batch; they are
        copied before this returns."""
        n = len(polys)
        if n == 0:
            return PendingBatch(self, 0, None, None, None)
        n, ptrs, degs_c, _keep = _marshal(polys, degrees)
        outs = (Factors * n)()
        sts = (C.c_int * n)()
        t = C.c_uint64(0)
        rc = lib().rfr_factor_batch_async(self._h, n, ptrs, degs_c, outs, sts, C.byref(t))
        if rc != RFR_OK:
            raise RFRError(rc, "rfr_factor_batch_async")
        self._inflight[t.value] = (outs, sts, n)
        return PendingBatch(self, n, outs, sts, t.value)

    def factor_batch_sharded(self, polys: Sequence[Sequence[int]], shard: int, nshards: int, gather) -> List[Result]:
        """This process's key-range shard of the batch (rfr_factor_batch_sharded).
        gather(list of (item, lo, hi)) -> every shard's triples, e.g.
        sharding.torch_gather(); None with one shard."""
        if gather is None:
            gather = list

        def _cb(mine, n_mine, all_pp, n_all_p, user):
            try:
                triples = [(int(mine[3 * i]), int(mine[3 * i + 1]), int(mine[3 * i + 2])) for i in range(n_mine)]
                allt = list(gather(triples))
                buf = _libc.malloc(max(1, 24 * len(allt)))
                if not buf:
                    return 1
                arr = (C.c_uint64 * max(1, 3 * len(allt))).from_address(buf)
                for i, (it, lo, hi) in enumerate(allt):
                    arr[3 * i], arr[3 * i + 1], arr[3 * i + 2] = it, lo, hi
                all_pp[0] = C.cast(buf, C.POINTER(C.c_uint64))
                n_all_p[0] = len(allt)
                return 0
            except Exception:
                return 1
        cb = GATHER_FN(_cb)
        n = len(polys)
        arrs = [_coeff_array(p) for p in polys]
        ptrs = (C.POINTER(C.c_int64) * n)(*[C.cast(a, C.POINTER(C.c_int64)) for a in arrs])
        degs = (C.c_int * n)(*[len(p) - 1 for p in polys])
        outs = (Factors * n)()
        sts = (C.c_int * n)()
        rc = lib().rfr_factor_batch_sharded(self._h, n, ptrs, degs, int(shard), int(nshards), cb, None, outs, sts)
        if rc != RFR_OK:
            lib().rfr_factors_free_n(outs, n)
            raise RFRError(rc, "rfr_factor_batch_sharded")
        return _to_results(n, sts, outs)

    def factor_batch_device(self, coeffs, degrees) -> List[Result]:
        """coeffs: int64 cuda tensor [count, 129] (ascending rows); degrees:
        int32 cuda tensor [count].  Inputs stay in device memory."""
        n = int(coeffs.shape[0])
        outs = (Factors * n)()
        sts = (C.c_int * n)()
        rc = lib().rfr_factor_batch_device(self._h, n, C.c_void_p(coeffs.data_ptr()),
                                           C.c_void_p(degrees.data_ptr()), outs, sts)
        if rc != RFR_OK:
            lib().rfr_factors_free_n(outs, n)
            raise RFRError(rc, "rfr_factor_batch_device")
        return _to_results(n, sts, outs)

    def submit(self, coeffs) -> int:
        """Queue one polynomial (a sequence of ints, or an int64 ctypes array made
        beforehand, which saves the conversion on the request path)."""
        t = C.c_uint64()
        arr = coeffs if isinstance(coeffs, C.Array) else _coeff_array(coeffs)
        st = lib().rfr_submit(self._h, arr, len(coeffs) - 1, C.byref(t))
        if st != RFR_OK:
            raise RFRError(st, "rfr_submit")
        return int(t.value)

    def poll(self, ticket: int) -> Optional[Result]:
        f = Factors()
        st = lib().rfr_poll(self._h, ticket, C.byref(f))
        if st == RFR_PENDING:
            return None
        if st == -1 and f.n_factors == 0 and not f.degrees:
            raise RFRError(st, "rfr_poll")
        return _to_result(st, f)

    def poll_batch(self, tickets: Sequence[int]) -> List[Optional[Result]]:
        """rfr_poll_batch: None for each request still pending."""
        n = len(tickets)
        if n == 0:
            return []
        ts = (C.c_uint64 * n)(*tickets)
        outs = (Factors * n)()
        sts = (C.c_int * n)()
        rc = lib().rfr_poll_batch(self._h, n, ts, outs, sts)
        if rc != RFR_OK:
            raise RFRError(rc, "rfr_poll_batch")
        return [None if sts[i] == RFR_PENDING else _to_result(sts[i], outs[i]) for i in range(n)]

    def wait(self, ticket: int, timeout_ms: int = -1) -> Result:
        f = Factors()
        st = lib().rfr_wait(self._h, ticket, timeout_ms, C.byref(f))
        if st == -12:
            raise RFRError(st, "rfr_wait")
        return _to_result(st, f)

    def cancel(self, ticket: int) -> int:
        return int(lib().rfr_cancel(self._h, ticket))


# ---------------------------------------------------------------- stages (torch tensors on CUDA)
def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(st, what):
    if st != RFR_OK:
        raise RFRError(st, what)


def stage_validate(coeffs, degrees):
    """Device input checks; returns status int32 [B] (RFR_OK, RFR_SF_SUSPECT = 2, or an error)."""
    import torch
    B = coeffs.shape[0]
    status = torch.zeros((B,), dtype=torch.int32, device=coeffs.device)
    _check(lib().rfr_stage_validate(_ptr(coeffs), _ptr(degrees), B, _ptr(status), _stream()), "rfr_stage_validate")
    return status


def stage_roots(coeffs, degrees, root_mode: int = RFR_ROOTS_FP64):
    """coeffs: int64 [B, 129] cuda; degrees: int32 [B] cuda.
    Returns (roots float64 [B, 128, 4], radius float64 [B, 128], status int32 [B])."""
    import torch
    B = coeffs.shape[0]
    roots = torch.zeros((B, RFR_MAX_DEGREE, 4), dtype=torch.float64, device=coeffs.device)
    radius = torch.zeros((B, RFR_MAX_DEGREE), dtype=torch.float64, device=coeffs.device)
    status = torch.zeros((B,), dtype=torch.int32, device=coeffs.device)
    _check(lib().rfr_stage_roots(_ptr(coeffs), _ptr(degrees), B, root_mode, _ptr(roots), _ptr(radius),
                                 _ptr(status), _stream()), "rfr_stage_roots")
    return roots, radius, status


def stage_weights(coeffs, degrees, roots, radius, status, eps_override: float = 0.0):
    """Returns the plans as a uint8 cuda tensor [B, sizeof(rfr_plan)] (view with PLAN_DTYPE)."""
    import torch
    B = coeffs.shape[0]
    plans = torch.zeros((B, PLAN_DTYPE.itemsize), dtype=torch.uint8, device=coeffs.device)
    _check(lib().rfr_stage_weights(_ptr(coeffs), _ptr(degrees), B, _ptr(roots), _ptr(radius), _ptr(status),
                                   eps_override, _ptr(plans), _stream()), "rfr_stage_weights")
    return plans


def stage_enumerate(w, h: int):
    """w: int64 cuda tensor holding uint64 weights bit-for-bit; returns keys int64 [2^h]."""
    import torch
    keys = torch.empty((1 << h,), dtype=torch.int64, device=w.device)
    _check(lib().rfr_stage_enumerate(_ptr(w), h, _ptr(keys), _stream()), "rfr_stage_enumerate")
    return keys


def match_workspace_bytes(n_a: int, n_b: int) -> int:
    return int(lib().rfr_stage_match_workspace(n_a, n_b))


def stage_match(w_a, w2_a, w_b, w2_b, window: int, window2: int, cap: int, exact: bool = False,
                fused: bool = False):
    """Weights as int64 cuda tensors (uint64 bits).  Returns (cand int64 [cap],
    counters int64 [6], workspace).  exact=True uses rfr_stage_match_exact
    (tables with the count-pass layout); fused=True uses rfr_stage_match_fused
    (no tables, any size it fits); otherwise rfr_stage_match chooses."""
    import torch
    n_a, n_b = int(w_a.numel()), int(w_b.numel())
    dev = w_b.device
    if fused:                                   # its own buffers, and room for fingerprint hits
        ws_bytes = int(lib().rfr_stage_match_fused_workspace(n_a, n_b))
        if ws_bytes == 0:
            raise RFRError(-1, f"the fused match does not take halves of {n_a} and {n_b} elements")
        ws_bytes += 8 * min(1 << (n_a + n_b), 1 << 26)
    else:
        ws_bytes = match_workspace_bytes(n_a, n_b)
    ws = torch.empty((ws_bytes // 8 + 64,), dtype=torch.int64, device=dev)
    base = ws.data_ptr()
    aligned = (base + 255) & ~255
    cand = torch.zeros((max(cap, 1),), dtype=torch.int64, device=dev)
    ctr = torch.zeros((6,), dtype=torch.int64, device=dev)
    fn = (lib().rfr_stage_match_exact if exact else
          lib().rfr_stage_match_fused if fused else lib().rfr_stage_match)
    _check(fn(_ptr(w_a) if n_a else None, _ptr(w2_a) if n_a else None, n_a,
                                 _ptr(w_b) if n_b else None, _ptr(w2_b) if n_b else None, n_b,
                                 int(window), int(window2), C.c_void_p(aligned), ws_bytes,
                                 _ptr(cand), int(cap), _ptr(ctr), _stream()), "rfr_stage_match")
    return cand, ctr, ws


def stage_lowlist(w, l: int, negate: bool = False):
    """Sorted low-subset list of the first l weights (int64 cuda tensor,
    uint64 bits): (sums int64 [2^l] ascending as uint64, masks int32 [2^l],
    workspace)."""
    import torch
    ws_bytes = int(lib().rfr_stage_lowlist_workspace(l))
    ws = torch.empty((ws_bytes // 8 + 64,), dtype=torch.int64, device=w.device)
    aligned = (ws.data_ptr() + 255) & ~255
    out = torch.empty((1 << l,), dtype=torch.int64, device=w.device)
    masks = torch.empty((1 << l,), dtype=torch.int32, device=w.device)
    _check(lib().rfr_stage_lowlist(_ptr(w) if l else None, l, int(bool(negate)), _ptr(out), _ptr(masks),
                                   C.c_void_p(aligned), ws_bytes, _stream()), "rfr_stage_lowlist")
    return out, masks, ws


def _splat_buffer(n_b: int, device):
    import torch
    cells = int(lib().rfr_stage_splat_cells(n_b))
    if cells == 0:
        raise RFRError(-1, f"splat: n_b = {n_b} out of range")
    return torch.empty((cells,), dtype=torch.int64, device=device), cells


def stage_splat(w_b, n_b: Optional[int] = None):
    """SPLAT of half b: (gamma int64 [cells] with the uint64 cells, counters int64 [8])."""
    import torch
    n_b = int(w_b.numel()) if n_b is None else n_b
    gamma, cells = _splat_buffer(n_b, w_b.device)
    ctr = torch.zeros((8,), dtype=torch.int64, device=w_b.device)
    _check(lib().rfr_stage_splat(_ptr(w_b) if n_b else None, n_b, _ptr(gamma), cells, _ptr(ctr), _stream()),
           "rfr_stage_splat")
    return gamma, ctr


def stage_splat_match(w_a, w2_a, w_b, w2_b, window: int, window2: int, cap: int):
    """Splat match (Algorithm E with the band query): (cand int64 [cap],
    counters int64 [8], gamma)."""
    import torch
    n_a, n_b = int(w_a.numel()), int(w_b.numel())
    gamma, cells = _splat_buffer(n_b, w_b.device)
    cand = torch.zeros((max(cap, 1),), dtype=torch.int64, device=w_b.device)
    ctr = torch.zeros((8,), dtype=torch.int64, device=w_b.device)
    _check(lib().rfr_stage_splat_match(_ptr(w_a) if n_a else None, _ptr(w2_a) if n_a else None, n_a,
                                       _ptr(w_b) if n_b else None, _ptr(w2_b) if n_b else None, n_b,
                                       int(window), int(window2), _ptr(gamma), cells, _ptr(cand), int(cap),
                                       _ptr(ctr), _stream()), "rfr_stage_splat_match")
    return cand, ctr, gamma


def stage_prune(w, w2, window: int, window2: int, cap: int):
    """Algorithm B over the m = len(w) elements: (cand int64 [cap], counters int64 [8])."""
    import torch
    m = int(w.numel())
    dev = w.device
    ws = torch.empty((64,), dtype=torch.int64, device=dev)
    aligned = (ws.data_ptr() + 255) & ~255
    cand = torch.zeros((max(cap, 1),), dtype=torch.int64, device=dev)
    ctr = torch.zeros((8,), dtype=torch.int64, device=dev)
    _check(lib().rfr_stage_prune(_ptr(w) if m else None, _ptr(w2) if m else None, m, int(window), int(window2),
                                 _ptr(cand), int(cap), _ptr(ctr), C.c_void_p(aligned), 256, _stream()),
           "rfr_stage_prune")
    return cand, ctr, ws


def stage_verify(coeffs, degrees, roots, plans, prob, pat_lo, pat_hi, want_coeffs: bool = False):
    import torch
    J = int(prob.numel())
    res = torch.zeros((J,), dtype=torch.int32, device=coeffs.device)
    co = torch.zeros((J, RFR_LDC), dtype=torch.int64, device=coeffs.device) if want_coeffs else None
    _check(lib().rfr_stage_verify(_ptr(coeffs), _ptr(degrees), _ptr(roots), _ptr(plans), _ptr(prob),
                                  _ptr(pat_lo), _ptr(pat_hi), J, _ptr(res), _ptr(co) if co is not None else None,
                                  _stream()), "rfr_stage_verify")
    return res, co
