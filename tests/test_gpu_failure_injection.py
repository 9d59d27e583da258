"""Failure injection on the host: a device allocator that fails on its i-th call.

mz_build and mz_build_batch route every device buffer of a plan (and the device
build's scratch) through the optional dev_alloc / dev_free callbacks. A callback
that returns NULL on its i-th call, for every i a build makes, must give
MZ_ERR_OOM with *out set to NULL and every buffer handed out so far returned:
the allocator's live bytes come back to where they started. No GPU fault is
involved; the failure is made on the host.
"""
import ctypes

import numpy as np
import pytest
import torch

import posetgen as pg
import paper_2211_13706_gb300 as mz

pytestmark = pytest.mark.gpu


class FailingAllocator:
    """dev_alloc / dev_free over torch's caching allocator that fails on call `fail_at`
    (0-based; -1 never fails) and tracks the bytes it has handed out."""

    def __init__(self, fail_at=-1):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.alloc_cb = mz._ALLOC_T(self._alloc)
        self.free_cb = mz._FREE_T(self._free)

    def _alloc(self, nbytes, ctx):
        i = self.calls
        self.calls += 1
        if i == self.fail_at:
            return None
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes))
        self.live[ptr] = int(nbytes)
        return ptr

    def _free(self, ptr, ctx):
        self.live.pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    def opts(self, **kw):
        o = mz._opts(kw.get("build_transpose", 0), 0, 0, 0, 0, kw.get("niv_format", 0), 0, 0,
                     kw.get("device_build", 0), False)
        o.dev_alloc = ctypes.cast(self.alloc_cb, ctypes.c_void_p).value
        o.dev_free = ctypes.cast(self.free_cb, ctypes.c_void_p).value
        return o


def _build(p, alloc, **kw):
    """mz_build through the C ABI; returns (status, the plan pointer it left in *out)."""
    src = np.ascontiguousarray(p.src, np.int32)
    dst = np.ascontiguousarray(p.dst, np.int32)
    cid = None if p.chain_id is None else np.ascontiguousarray(p.chain_id, np.int32)
    opts = alloc.opts(**kw)
    out = ctypes.c_void_p(0xDEAD)                 # must come back NULL on an error
    st = mz.lib.mz_build(p.n, src.size, src.ctypes.data, dst.ctypes.data,
                         None if cid is None else cid.ctypes.data, ctypes.byref(opts), ctypes.byref(out))
    return st, out.value


def _build_batch(ps, alloc, **kw):
    count = len(ps)
    ns = np.array([p.n for p in ps], np.int64)
    srcs = [np.ascontiguousarray(p.src, np.int32) for p in ps]
    dsts = [np.ascontiguousarray(p.dst, np.int32) for p in ps]
    ms = np.array([a.size for a in srcs], np.int64)
    arr = lambda xs: (ctypes.c_void_p * count)(*[a.ctypes.data for a in xs])
    opts = alloc.opts(**kw)
    out = ctypes.c_void_p(0xDEAD)
    st = mz.lib.mz_build_batch(count, ns.ctypes.data, ms.ctypes.data, arr(srcs), arr(dsts), None,
                               ctypes.byref(opts), ctypes.byref(out))
    return st, out.value


CASES = {
    "dense": dict(poset=lambda: pg.planted_chain_poset(3000, 12, 3, cross_deg=2), kw=dict(build_transpose=1)),
    "sparse": dict(poset=lambda: pg.planted_chain_poset(2000, 40, 4, cross_deg=2), kw=dict(niv_format=2)),
    "device_build": dict(poset=lambda: pg.planted_chain_poset(3000, 12, 5, cross_deg=2),
                         kw=dict(device_build=1, build_transpose=1)),
    "device_build_sparse": dict(poset=lambda: pg.planted_chain_poset(2000, 40, 6, cross_deg=2),
                                kw=dict(device_build=1, niv_format=2)),
    # chains by Alg. 1's matching on the device (the ER DAG comes without chains)
    "device_build_matching": dict(poset=lambda: pg.er_dag(3000, 3, 7), kw=dict(device_build=2)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_every_allocation_failure_is_oom_without_leaks(case):
    p = CASES[case]["poset"]()
    kw = CASES[case]["kw"]
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    counter = FailingAllocator()
    st, plan = _build(p, counter, **kw)
    assert st == mz.MZ_OK and plan
    total = counter.calls
    assert total >= 5 and counter.live
    mz.lib.mz_destroy(plan)
    assert not counter.live and torch.cuda.memory_allocated() == base
    for i in range(total):
        a = FailingAllocator(fail_at=i)
        st, out = _build(p, a, **kw)
        assert st == mz.MZ_ERR_OOM, (case, i, mz._status_string(st), mz.lib.mz_last_error())
        assert out is None, (case, i)
        assert not a.live, (case, i, len(a.live))
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base, (case, i)


def test_batch_build_allocation_failures():
    ps = [pg.planted_chain_poset(800, 6, 7, cross_deg=2), pg.paper_example(), pg.boolean_lattice(5)]
    base = torch.cuda.memory_allocated()
    counter = FailingAllocator()
    st, plan = _build_batch(ps, counter)
    assert st == mz.MZ_OK
    mz.lib.mz_destroy(plan)
    for i in range(counter.calls):
        a = FailingAllocator(fail_at=i)
        st, out = _build_batch(ps, a)
        assert st == mz.MZ_ERR_OOM and out is None and not a.live, (i, mz._status_string(st))
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_callback_error_other_than_oom_is_raised_not_reported_as_oom(monkeypatch):
    """The binding's torch allocator maps only an allocation failure to MZ_ERR_OOM; any
    other exception inside the callback surfaces as that exception."""
    p = pg.planted_chain_poset(500, 4, 8, cross_deg=2)

    def broken(nbytes):
        raise ValueError("not an out-of-memory error")

    monkeypatch.setattr(torch.cuda, "caching_allocator_alloc", broken)
    with pytest.raises(RuntimeError, match="allocation callback failed"):
        mz.Plan(p.n, p.src, p.dst, p.chain_id, torch_allocator=True)

    def oom(nbytes):
        raise torch.cuda.OutOfMemoryError("injected")

    monkeypatch.setattr(torch.cuda, "caching_allocator_alloc", oom)
    with pytest.raises(mz.MzError) as e:
        mz.Plan(p.n, p.src, p.dst, p.chain_id, torch_allocator=True)
    assert e.value.status == mz.MZ_ERR_OOM
