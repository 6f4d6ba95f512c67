"""Host-buffer entry points: a build from host keys equals the device build,
and a chunked, overlapped host lookup equals the device lookup and the
oracle, for pinned and pageable buffers, int32 and int64 values, needle
counts around the chunk size and NULL outputs."""
import numpy as np
import pytest

import oracle as O
from paper_2508_11443_b300 import workloads as W

pytestmark = pytest.mark.gpu
CHUNK = 1 << 23


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


@pytest.mark.parametrize("n,nq", [(1, 1), (1000, 3), (70000, CHUNK + 5), (1 << 20, 2 * CHUNK), (4096, 3 * CHUNK + 17)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_build_and_lookup(F, n, nq, pinned):
    import torch
    w = W.u64_workload(n, nq, 0.6, seed=n + nq)
    keys, vals, q = w.keys, w.vals, w.queries
    if pinned:
        keys = torch.from_numpy(keys.view(np.int64)).pin_memory()
        vals = torch.from_numpy(vals).pin_memory()
        q = torch.from_numpy(q.view(np.int64)).pin_memory()
        out = torch.empty(nq, dtype=torch.int64).pin_memory()
        found = torch.empty(nq, dtype=torch.uint8).pin_memory()
    else:
        out = np.empty(nq, np.int64)
        found = np.empty(nq, np.uint8)
    hm = F.fks_build_u64_host(keys, vals, 7)
    dm = F.fks_build_u64(dev(w.keys), dev(w.vals), 7)
    hd, hs, _ = F.fks_map_export(hm)
    dd, ds, _ = F.fks_map_export(dm)
    assert np.array_equal(hd, dd) and np.array_equal(hs, ds)
    F.fks_lookup_u64_host(hm, q, out, found, -9)
    o = out.numpy() if pinned else out
    f = found.numpy() if pinned else found
    assert np.array_equal(f, w.expect_found)
    assert np.array_equal(o, np.where(w.expect_found == 1, w.expect_vals, -9))
    if n <= 70000:
        om = O.build_u64(w.keys, w.vals, seed=7)
        oo, of = O.lookup_u64(om, w.queries[:100000], absent=-9)
        assert np.array_equal(o[:100000], oo) and np.array_equal(f[:100000], of)


def test_host_int32_and_null_outputs(F):
    w = W.u64_workload(5000, CHUNK + 1000, 0.5, seed=3)
    vals = (np.arange(5000) - 77).astype(np.int32)
    m = F.fks_build_u64_host(w.keys, vals, 11)
    out = np.empty(w.queries.size, np.int32)
    F.fks_lookup_u64_host(m, w.queries, out, None, -1)
    assert np.array_equal(out.astype(np.int64), np.where(w.expect_found == 1, w.expect_vals - 77, -1))
    found = np.empty(w.queries.size, np.uint8)
    F.fks_lookup_u64_host(m, w.queries, None, found, -1)
    assert np.array_equal(found, w.expect_found)


def test_host_lookup_rejects_string_maps(F):
    s = W.string_workload(100, 10, 0.5, seed=1)
    m = F.fks_build_bytes(dev(s.ctx), dev(s.offs), dev(s.vals), 1)
    with pytest.raises(F.FksError) as e:
        F.fks_lookup_u64_host(m, np.zeros(4, np.uint64), np.empty(4, np.int64), None, -1)
    assert e.value.status == F.FKS_ERR_INVALID_ARG
