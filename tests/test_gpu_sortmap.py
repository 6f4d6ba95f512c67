"""The search-based comparison map (mk_arraymap, Sec. 3.4): the device radix
sort must equal a stable library sort of the pairs, and lookups must equal a
lower-bound binary search (numpy searchsorted, which the oracle's own binary
search is pinned against)."""
import numpy as np
import pytest

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


def expected(keys, vals, q, absent):
    order = np.argsort(keys, kind="stable")
    sk, sv = keys[order], vals[order]
    i = np.searchsorted(sk, q, side="left")
    hit = (i < sk.size) & (sk[np.minimum(i, sk.size - 1)] == q)
    return sk, sv, np.where(hit, sv[np.minimum(i, sk.size - 1)], absent), hit.astype(np.uint8)


@pytest.mark.parametrize("n", [1, 7, 2047, 2048, 2049, 100000, (1 << 20) + 3])
def test_sort_and_search(F, n):
    import torch
    w = W.u64_workload(n, 2 * n, 0.5, seed=n + 1)
    m = F.fks_sortmap_build(dev(w.keys), dev(w.vals))
    sk, sv = F.fks_sortmap_export(m)
    ek, ev, eo, ef = expected(w.keys, w.vals, w.queries, -4)
    assert np.array_equal(sk, ek) and np.array_equal(sv, ev)
    out = torch.empty(w.queries.size, dtype=torch.int64, device="cuda")
    found = torch.empty(w.queries.size, dtype=torch.uint8, device="cuda")
    F.fks_sortmap_lookup(m, dev(w.queries), out, found, -4)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), eo) and np.array_equal(found.cpu().numpy(), ef)


def test_sort_is_stable_and_int32_values(F):
    import torch
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 50, 30000).astype(np.uint64) * np.uint64(0x0101010101010101)
    vals = np.arange(keys.size, dtype=np.int32)
    m = F.fks_sortmap_build(dev(keys), dev(vals))
    sk, sv = F.fks_sortmap_export(m)
    ek, ev, _, _ = expected(keys, vals.astype(np.int64), keys[:10], -1)
    assert np.array_equal(sk, ek) and np.array_equal(sv, ev)  # equal keys keep input order
    out = torch.empty(100, dtype=torch.int32, device="cuda")
    F.fks_sortmap_lookup(m, dev(keys[:100]), out, None, -1)
    torch.cuda.synchronize()
    _, _, eo, _ = expected(keys, vals.astype(np.int64), keys[:100], -1)
    assert np.array_equal(out.cpu().numpy().astype(np.int64), eo)


# ------------------------------------------------------------------ Eytzinger layout (Sec. 3.4)
@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 1023, 1024, 2049, 100000, (1 << 20) + 3, (1 << 22) + 12345])
def test_eytzinger_layout_and_search(F, n):
    """The device layout equals the oracle's Eytzinger layout of the sorted
    pairs; lookups equal the oracle's Eytzinger search and binary search."""
    import torch
    import oracle as O
    w = W.u64_workload(n, 2 * n + 2, 0.5, seed=n + 9)
    m = F.fks_eytzmap_build(dev(w.keys), dev(w.vals))
    gk, gv = F.fks_sortmap_export(m)
    sk, sv, eo, ef = expected(w.keys, w.vals, w.queries, -4)
    ok, ov = O.eytzinger_layout(sk, sv)
    assert np.array_equal(gk, ok[1:]) and np.array_equal(gv, ov[1:])
    q = np.concatenate([w.queries, [0, 2**64 - 1], sk[:1], sk[-1:]]).astype(np.uint64)
    out = torch.empty(q.size, dtype=torch.int64, device="cuda")
    found = torch.empty(q.size, dtype=torch.uint8, device="cuda")
    F.fks_sortmap_lookup(m, dev(q), out, found, -4)
    torch.cuda.synchronize()
    _, _, eo, ef = expected(w.keys, w.vals, q, -4)
    assert np.array_equal(out.cpu().numpy(), eo) and np.array_equal(found.cpu().numpy(), ef)
    for x in q[:: max(1, q.size // 500)].tolist():  # the oracle's own search on a sample
        k = O.eytzinger_search(ok, x)
        i = int(np.searchsorted(sk, x))
        assert (k != 0) == (i < sk.size and sk[min(i, sk.size - 1)] == x)


def test_eytzinger_int32_values(F):
    import torch
    w = W.u64_workload(5000, 3000, 0.5, seed=4)
    vals = np.arange(5000, dtype=np.int32) - 2500
    m = F.fks_eytzmap_build(dev(w.keys), dev(vals))
    out = torch.empty(3000, dtype=torch.int32, device="cuda")
    F.fks_sortmap_lookup(m, dev(w.queries), out, None, -7)
    torch.cuda.synchronize()
    _, _, eo, _ = expected(w.keys, vals.astype(np.int64), w.queries, -7)
    assert np.array_equal(out.cpu().numpy().astype(np.int64), eo)
