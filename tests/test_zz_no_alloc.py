"""The allocation-free match entry point, checked against the regular one.

rfr_stage_match_noalloc serves callers that cannot allocate device memory
(a host framework that owns all of it, or a loop where an allocation that may
synchronise the device is not allowed).  It must produce exactly what
rfr_stage_match produces with a caller-provided workspace, call after call,
although every call reuses the same fixed scratch array inside the library.
This file is collected last on purpose."""
import ctypes
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M64 = 1 << 64


def _u64(vals):
    a = np.asarray([int(v) for v in vals], dtype=np.uint64).view(np.int64)
    return torch.from_numpy(a.copy()).cuda()


def _weights(seed, na, nb):
    rng = random.Random(seed)
    wa = [rng.randrange(M64) for _ in range(na)]
    wb = [rng.randrange(M64) for _ in range(nb)]
    wb[1] = (-(wa[0] + wa[3] + wb[4])) % M64          # planted integral subsets
    wa[5] = (-(wb[2] + wb[6])) % M64
    w2a = [rng.randrange(1 << 20) for _ in range(na)]
    w2b = [rng.randrange(1 << 20) for _ in range(nb)]
    return wa, w2a, wb, w2b


def _noalloc(L, t, window, window2, cap):
    wa, w2a, wb, w2b = t
    cand = torch.zeros((cap,), dtype=torch.int64, device="cuda")
    ctr = torch.zeros((6,), dtype=torch.int64, device="cuda")
    st = L.rfr_stage_match_noalloc(ctypes.c_void_p(wa.data_ptr()), ctypes.c_void_p(w2a.data_ptr()), wa.numel(),
                                   ctypes.c_void_p(wb.data_ptr()), ctypes.c_void_p(w2b.data_ptr()), wb.numel(),
                                   window, window2, ctypes.c_void_p(cand.data_ptr()), cap,
                                   ctypes.c_void_p(ctr.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, cand, ctr


def _result(cand, ctr, cap):
    c = ctr.cpu().numpy().view(np.uint64)
    n = int(c[2])
    return sorted(int(x) for x in cand.cpu().numpy().view(np.uint64)[:min(n, cap)]), [int(x) for x in c[:5]]


# (12, 13): the shared-memory match; (16, 17): the fused match; (12, 16): the
# table match, whose bucket cursors and halo counts must start at zero.  It
# runs after the fused call, so the shared array still holds that call's data.
@pytest.mark.parametrize("seed,na,nb", [(31, 12, 13), (32, 16, 17), (33, 12, 16)])
def test_noalloc_matches_regular_entry_twice(seed, na, nb):
    import paper_2410_15880_b300 as P
    L = P.lib()
    wa, w2a, wb, w2b = _weights(seed, na, nb)
    t = (_u64(wa), _u64(w2a), _u64(wb), _u64(w2b))
    window, window2, cap = 1 << 40, 1 << 62, 1 << 12
    cand, ctr, _ws = P.stage_match(t[0], t[1], t[2], t[3], window, window2, cap)
    torch.cuda.synchronize()
    expect = _result(cand, ctr, cap)
    assert len(expect[0]) >= 2                      # the planted subsets are found
    for _ in range(2):                              # two calls in a row share the scratch array
        st, c2, k2 = _noalloc(L, t, window, window2, cap)
        assert st == 0
        assert _result(c2, k2, cap) == expect


def test_noalloc_rejects_too_large_halves():
    import paper_2410_15880_b300 as P
    L = P.lib()
    t = tuple(_u64([1] * 24) for _ in range(4))
    st, _, _ = _noalloc(L, t, 1 << 40, 1 << 62, 16)
    assert st == -11                               # RFR_E_BUDGET: beyond the fixed scratch
