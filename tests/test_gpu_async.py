"""Asynchronous builds: the handle returned at once reports, through
fks_map_info, the status the blocking build would have returned, and its
tables equal the blocking build's; lookups, export and destroy wait for the
build.  Batched builds accept segment offsets in device memory."""
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


@pytest.mark.parametrize("n", [1, 5000, (1 << 20) + 9])
def test_async_equals_blocking(F, n):
    import torch
    w = W.u64_workload(n, 4 * n + 1, 0.5, seed=n)
    keys, vals = dev(w.keys), dev(w.vals)
    handles = [F.fks_build_u64_async(keys, vals, 3 + i) for i in range(3)]  # several in flight
    for i, h in enumerate(handles):
        assert F.fks_map_status(h) == F.FKS_OK
        b = F.fks_build_u64(keys, vals, 3 + i)
        da, sa, _ = F.fks_map_export(h)
        db, sb, _ = F.fks_map_export(b)
        assert np.array_equal(da, db) and np.array_equal(sa, sb)
    om = O.build_u64(w.keys, w.vals, seed=3)
    da, sa, _ = F.fks_map_export(handles[0])
    assert np.array_equal(da, om.desc) and np.array_equal(sa, om.slots)


def test_lookup_waits_for_the_build(F):
    import torch
    w = W.u64_workload(1 << 21, 1 << 20, 0.5, seed=4)
    keys, vals = dev(w.keys), dev(w.vals)  # inputs stay alive until the build is done
    h = F.fks_build_u64_async(keys, vals, 9)
    out = torch.empty(w.queries.size, dtype=torch.int64, device="cuda")
    found = torch.empty(w.queries.size, dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(h, dev(w.queries), out, found, -1)  # issued while the build may still run
    torch.cuda.synchronize()
    assert np.array_equal(found.cpu().numpy(), w.expect_found)
    assert np.array_equal(out.cpu().numpy(), np.where(w.expect_found == 1, w.expect_vals, -1))


def test_async_failure_is_reported(F):
    import torch
    keys = np.concatenate([W.key_stream(5, 1000), W.key_stream(5, 3)]).astype(np.uint64)
    dk, dv = dev(keys), dev(np.arange(keys.size))
    h = F.fks_build_u64_async(dk, dv, 1)
    assert F.fks_map_status(h) == F.FKS_ERR_DUPLICATE_KEY
    with pytest.raises(F.FksError) as e:
        F.fks_lookup_u64(h, dev(keys[:4]), torch.empty(4, dtype=torch.int64, device="cuda"), None, -1)
    assert e.value.status == F.FKS_ERR_DUPLICATE_KEY
    del h  # destroy of a failed handle


def test_destroy_while_building(F):
    w = W.u64_workload(1 << 20, 10, 0.5, seed=6)
    keys, vals = dev(w.keys), dev(w.vals)
    for i in range(4):
        h = F.fks_build_u64_async(keys, vals, i)
        del h  # joins the build, frees its tables


def test_async_strings(F):
    w = W.string_workload(20000, 100, 0.5, seed=7)
    ctx, offs, vals = dev(w.ctx), dev(w.offs), dev(w.vals)
    h = F.fks_build_bytes_async(ctx, offs, vals, 5)
    assert F.fks_map_status(h) == F.FKS_OK
    om = O.build_bytes(w.ctx, w.offs, w.vals, seed=5)
    d, s_, _ = F.fks_map_export(h)
    assert np.array_equal(d, om.desc) and np.array_equal(s_, om.slots)


def test_batched_device_segment_offsets(F):
    b = W.batched_workload(9, 1, 5000, 100, 0.75, seed=8)
    a = F.fks_build_batched(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, b.seeds, dev(b.vals))
    c = F.fks_build_batched(F.FKS_KEY_U64, dev(b.keys), None, None, dev(b.seg_offs), b.seeds, dev(b.vals))
    for j in range(9):
        d1, s1, _ = F.fks_map_export(a.get(j))
        d2, s2, _ = F.fks_map_export(c.get(j))
        assert np.array_equal(d1, d2) and np.array_equal(s1, s2)
