"""Failure paths of the host runtime, made on the host: a memory budget too
small for one problem's tables, an allocator that cannot allocate, PyTorch's
caching allocator as the context's allocator, and one context per GPU in a
process.  Nothing here faults or hangs a GPU: the failures are returned
statuses, and every other problem of the batch must still be exact."""
import pytest

from gpu_util import golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RFR_E_OOM = -10
RFR_E_BUDGET = -11


def _batch():
    """A degree-100 problem (tables of tens of MB) between two small ones."""
    recs = [golden("cfg2")[0], golden("cfg3")[0], golden("cfg1")[0]]
    return recs, [r["coeffs"] for r in recs]


def test_budget_smaller_than_one_problem_fails_only_that_problem():
    from paper_2410_15880_b300 import Context
    recs, polys = _batch()
    with Context(device=0, mem_budget_bytes=8 << 20) as c:
        res = c.factor_batch(polys)
        assert res[1].status == RFR_E_BUDGET
        for i in (0, 2):
            assert res[i].ok and res[i].factors == recs[i]["factors"]
    with Context(device=0) as c:                     # the default budget takes it
        res = c.factor_batch(polys)
        assert all(r.ok for r in res) and [r.factors for r in res] == [r["factors"] for r in recs]


class _Armed:
    """PyTorch's caching allocator behind a switch: while armed, every request
    of more than `limit` bytes returns 0 (no memory)."""

    def __init__(self, limit):
        self.limit, self.armed, self.refused, self.live = limit, False, 0, {}

    def alloc(self, nbytes, stream):
        if self.armed and nbytes > self.limit:
            self.refused += 1
            return 0
        p = torch.cuda.caching_allocator_alloc(nbytes, 0, stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, nbytes, stream):
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)


def test_allocator_without_memory_gives_oom_then_recovers():
    """Requests beyond 4 MB fail while the allocator is armed: the degree-100
    problem ends with RFR_E_OOM (the small ones are exact), nothing the call
    allocated stays allocated, and the next call with memory succeeds."""
    from paper_2410_15880_b300 import Context, RFRError
    recs, polys = _batch()
    A = _Armed(4 << 20)
    with Context(device=0) as c:
        c.set_allocator(A.alloc, A.free)
        res = c.factor_batch(polys)                  # warm: the context's own buffers are made
        assert all(r.ok for r in res)
        kept = dict(A.live)
        A.armed = True
        try:
            res = c.factor_batch(polys)
            assert res[1].status == RFR_E_OOM
            for i in (0, 2):
                assert res[i].ok and res[i].factors == recs[i]["factors"]
        except RFRError as e:                        # a failure outside one problem's tables
            assert e.status == RFR_E_OOM
        assert A.refused >= 1
        assert A.live == kept                        # no leak
        A.armed = False
        res = c.factor_batch(polys)
        assert all(r.ok for r in res) and [r.factors for r in res] == [r["factors"] for r in recs]
    assert A.live == {}                              # rfr_destroy returned everything


def test_torch_caching_allocator_batch_equals_goldens():
    from paper_2410_15880_b300 import Context
    recs = golden("cfg2")[:6] + golden("cfg3")[:2] + golden("cfg1")
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated(0)
    with Context(device=0) as c:
        c.use_torch_allocator()
        res = c.factor_batch([r["coeffs"] for r in recs])
        assert all(r.ok for r in res)
        assert [r.factors for r in res] == [r["factors"] for r in recs]
        assert torch.cuda.memory_allocated(0) > base  # the context's buffers came from torch
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(0) == base


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two visible GPUs")
def test_one_context_per_device_in_one_process():
    """Kernel attributes (large shared memory) are set per device: the same
    degree-100 problem factors through contexts on device 0 and device 1."""
    from paper_2410_15880_b300 import Context
    r = golden("cfg3")[0]
    for dev in (0, 1):
        with torch.cuda.device(dev), Context(device=dev) as c:
            res = c.factor(r["coeffs"])
            assert res.ok and res.factors == r["factors"]
