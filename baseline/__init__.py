"""CPU baselines timed beside the GPU path (not part of it).

hs_mt: a multithreaded C++ Horowitz–Sahni band join (enumerate, parallel
LSD radix sort, partitioned join) over all host cores: the match stage of
Section 3.3 on the CPU.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hs_mt.cpp")
LIB = os.path.join(HERE, "libhs_mt.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile libhs_mt.so with g++ (generic x86-64 code: the library is built
    on one host and may run on another)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-pthread", SRC, "-o", LIB],
                       check=True)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        u64p = C.POINTER(C.c_uint64)
        L.hs_mt_match.restype = C.c_int
        L.hs_mt_match.argtypes = [u64p, u64p, C.c_int, u64p, u64p, C.c_int, C.c_uint64, C.c_uint64,
                                  C.c_int, u64p, C.c_uint64, u64p, C.POINTER(C.c_double)]
        _lib = L
    return _lib


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


def hs_mt_match(w_a, w2_a, w_b, w2_b, window: int, window2: int, threads: int = 0, cap: int = 1 << 16):
    """Weights as sequences of uint64 ints.  Returns (candidates as a list of
    patterns s_a | s_b << n_a, counts (pairs within W, candidates, trivial
    seen), seconds (enumerate, sort, join))."""
    import numpy as np
    u64p = C.POINTER(C.c_uint64)
    arr = [np.ascontiguousarray(np.asarray([int(x) for x in v], dtype=np.uint64).reshape(-1))
           for v in (w_a, w2_a, w_b, w2_b)]
    arr = [x if x.size else np.zeros(1, dtype=np.uint64) for x in arr]
    out = np.zeros(max(cap, 1), dtype=np.uint64)
    counts = np.zeros(3, dtype=np.uint64)
    secs = (C.c_double * 3)()
    st = lib().hs_mt_match(arr[0].ctypes.data_as(u64p), arr[1].ctypes.data_as(u64p), len(w_a),
                           arr[2].ctypes.data_as(u64p), arr[3].ctypes.data_as(u64p), len(w_b),
                           int(window), int(window2), int(threads or host_cores()),
                           out.ctypes.data_as(u64p), cap, counts.ctypes.data_as(u64p), secs)
    if st != 0:
        raise ValueError(f"hs_mt_match: invalid arguments (status {st})")
    n = int(min(int(counts[1]), cap))
    return [int(x) for x in out[:n]], [int(x) for x in counts], list(secs)
