"""The device-memory hook (fks_allocator): every byte a build keeps comes from
the caller's allocator and goes back to it when the map is destroyed; an
allocation that fails at any point of a build is reported as
FKS_ERR_OUT_OF_MEMORY and leaves nothing allocated (failure injected on the
host, by the hook returning NULL)."""
import gc

import numpy as np
import pytest

import oracle as O
from paper_2508_11443_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch  # noqa: F401
    from paper_2508_11443_b300 import build, fks
    build.build()
    return fks


def dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


class Counting:
    """Torch's caching allocator behind a ledger; fail_at = the n-th call
    returns NULL."""

    def __init__(self, F, fail_at=None):
        import torch
        self.torch = torch
        self.live, self.calls, self.fail_at, self.problems = {}, 0, fail_at, []
        self.hook = F.Allocator(self.alloc, self.free)

    def alloc(self, n, stream):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(n, stream=stream)
        self.live[p] = n
        return p

    def free(self, p, n, stream):
        if self.live.pop(p, None) != n:
            self.problems.append((p, n))
        self.torch.cuda.caching_allocator_delete(p)


def settle():
    import torch
    gc.collect()
    torch.cuda.synchronize()


def test_u64_and_string_maps_live_in_the_callers_memory(F):
    w = W.u64_workload((1 << 20) + 5, 5000, 0.5, seed=31)
    A = Counting(F)
    m = F.fks_build_u64(dev(w.keys), dev(w.vals), 4, alloc=A.hook)
    assert A.calls >= 2 and len(A.live) == 1  # the scratch went back, the tables stayed
    info = F.fks_map_info(m)
    assert list(A.live.values())[0] >= info.bytes
    d, s, _ = F.fks_map_export(m)
    om = O.build_u64(w.keys, w.vals, seed=4)
    assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots)
    del m
    settle()
    assert not A.live and not A.problems
    st = W.string_workload(20000, 100, 0.5, seed=32)
    m = F.fks_build_bytes(dev(st.ctx), dev(st.offs), dev(st.vals), 5, alloc=A.hook)
    assert len(A.live) == 1
    del m
    settle()
    assert not A.live and not A.problems


def test_batched_set_lives_in_the_callers_memory(F):
    b = W.batched_workload(20, 16, 5000, 1000, 0.75, seed=33)
    A = Counting(F)
    S = F.fks_build_batched(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, b.seeds, dev(b.vals), alloc=A.hook)
    assert len(A.live) == 2  # the set's tables and its lookup table
    del S
    settle()
    assert not A.live and not A.problems


@pytest.mark.parametrize("fail_at", [1, 2, 3, 4, 5])
def test_a_failed_allocation_leaks_nothing(F, fail_at):
    w = W.u64_workload((1 << 20) + 5, 10, 0.5, seed=34)
    keys, vals = dev(w.keys), dev(w.vals)
    A = Counting(F, fail_at=fail_at)
    try:
        m = F.fks_build_u64(keys, vals, 4, alloc=A.hook)
    except F.FksError as e:
        assert e.status == F.FKS_ERR_OUT_OF_MEMORY
        settle()
        assert not A.live and not A.problems
    else:  # fewer allocations than fail_at: a normal build
        assert A.calls < fail_at
        del m
        settle()
        assert not A.live
    # from_array: the deduplication pre-pass allocates first
    dup = np.concatenate([w.keys[:1000], w.keys[:1000]])
    A2 = Counting(F, fail_at=fail_at)
    try:
        m = F.fks_build_u64(dev(dup), dev(np.arange(2000)), 4, opts=F.make_opts(dedup=1), alloc=A2.hook)
    except F.FksError as e:
        assert e.status == F.FKS_ERR_OUT_OF_MEMORY
    else:
        del m
    settle()
    assert not A2.live and not A2.problems


def test_async_build_uses_the_hook_from_its_worker_thread(F):
    w = W.u64_workload(300000, 10, 0.5, seed=35)
    A = Counting(F)
    m = F.fks_build_u64_async(dev(w.keys), dev(w.vals), 6)
    assert F.fks_map_status(m) == F.FKS_OK
    del m
    L = F.lib()
    import ctypes
    h = ctypes.c_void_p()
    keys, vals = dev(w.keys), dev(w.vals)
    st = L.fks_build_u64_async(F._ptr(keys), F._ptr(vals), F.FKS_VAL_I64, keys.numel(), 6, None, A.hook.ref(),
                               F._stream(None), ctypes.byref(h))
    assert st == F.FKS_OK
    m = F.Map(h.value)
    assert F.fks_map_status(m) == F.FKS_OK and len(A.live) == 1
    del m
    settle()
    assert not A.live and not A.problems
