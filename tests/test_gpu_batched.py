"""Batched builds over segment descriptors: every map of a set equals a per-call
build of its segment with the same seed, byte for byte, and equals the oracle;
batched (map_id, key) lookups equal per-map lookups."""
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


def export(F, m):
    d, s, c = F.fks_map_export(m)
    return d, s


def batched_lookup(F, S, ids, q, i64=True):
    import torch
    out = torch.empty(len(q), dtype=torch.int64 if i64 else torch.int32, device="cuda")
    found = torch.empty(len(q), dtype=torch.uint8, device="cuda")
    F.fks_lookup_batched(S, dev(ids.astype(np.uint32)), q=dev(q), out_vals=out, out_found=found)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int64), found.cpu().numpy()


@pytest.mark.parametrize("m,lo,hi", [(1, 16, 16), (7, 1, 3000), (64, 16, 1 << 14)])
def test_batched_equals_per_call_and_oracle(F, m, lo, hi):
    b = W.batched_workload(m, lo, hi, 20000, 0.75, seed=4 + m)
    S = F.fks_build_batched(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, b.seeds, dev(b.vals))
    assert (S.status == 0).all() and len(S) == m
    for j in range(m):
        k = b.keys[b.seg_offs[j]:b.seg_offs[j + 1]]
        v = b.vals[b.seg_offs[j]:b.seg_offs[j + 1]]
        om = O.build_u64(k, v, seed=int(b.seeds[j]))
        d, s = export(F, S.get(j))
        assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots), j
        if j < 8:
            pm = F.fks_build_u64(dev(k), dev(v), int(b.seeds[j]))
            d2, s2 = export(F, pm)
            assert np.array_equal(d, d2) and np.array_equal(s, s2)
    out, found = batched_lookup(F, S, b.q_map, b.q_keys)
    assert np.array_equal(found, b.expect_found)
    assert np.array_equal(out, np.where(b.expect_found == 1, b.expect_vals, -1))


def test_batched_with_a_failing_map(F):
    b = W.batched_workload(5, 100, 2000, 5000, 0.75, seed=9)
    keys = b.keys.copy()
    s2 = b.seg_offs[2]
    keys[s2 + 1] = keys[s2]  # map 2 holds a duplicate
    with pytest.raises(F.FksError):
        F.fks_build_batched(F.FKS_KEY_U64, dev(keys), None, None, b.seg_offs, b.seeds, dev(b.vals))
    S = F.fks_build_batched(F.FKS_KEY_U64, dev(keys), None, None, b.seg_offs, b.seeds, dev(b.vals),
                            raise_on_error=False)
    assert S.status.tolist() == [0, 0, F.FKS_ERR_DUPLICATE_KEY, 0, 0]
    assert S.get(2) is None
    out, found = batched_lookup(F, S, b.q_map, b.q_keys)
    ok = b.q_map != 2
    assert np.array_equal(found[ok], b.expect_found[ok])
    assert not found[~ok].any()
    # an unknown map id is absent, never an out-of-range read
    out, found = batched_lookup(F, S, np.array([7, 99, 2**31], np.uint32), b.q_keys[:3])
    assert not found.any() and (out == -1).all()


def test_batched_strings(F):
    import torch
    parts = [W.string_workload(n, 10, 0.5, seed=50 + n) for n in (3, 700, 1, 2500)]
    ctx = np.concatenate([p.ctx for p in parts])
    offs = [np.zeros(1, np.int64)]
    base = 0
    for p in parts:
        offs.append(p.offs[1:] + base)
        base += p.offs[-1]
    offs = np.concatenate(offs)
    seg = np.cumsum([0] + [p.offs.size - 1 for p in parts])
    vals = np.concatenate([p.vals for p in parts]).astype(np.int32)
    seeds = np.array([11, 12, 13, 14], np.uint64)
    S = F.fks_build_batched(F.FKS_KEY_BYTES, None, dev(ctx), dev(offs), seg, seeds, dev(vals))
    for j, p in enumerate(parts):
        om = O.build_bytes(p.ctx, p.offs, p.vals, seed=int(seeds[j]))
        d, s = export(F, S.get(j))
        # slot offsets point into the set's shared context: shift the oracle's
        shift = np.uint64(offs[seg[j]])
        exp = om.slots.copy()
        exp[:, 1] += shift
        assert np.array_equal(d, om.desc) and np.array_equal(s, exp)
    # needles: each part's own query strings against its map id
    qctx = np.concatenate([p.qctx for p in parts])
    qo = [np.zeros(1, np.int64)]
    base = 0
    ids = []
    for j, p in enumerate(parts):
        qo.append(p.qoffs[1:] + base)
        base += p.qoffs[-1]
        ids += [j] * (p.qoffs.size - 1)
    qo = np.concatenate(qo)
    out = torch.empty(len(ids), dtype=torch.int32, device="cuda")
    found = torch.empty(len(ids), dtype=torch.uint8, device="cuda")
    F.fks_lookup_batched(S, dev(np.array(ids, np.uint32)), qctx=dev(qctx), qoffs=dev(qo), out_vals=out,
                         out_found=found)
    torch.cuda.synchronize()
    ef = np.concatenate([p.expect_found for p in parts])
    ev = np.concatenate([p.expect_vals for p in parts])
    assert np.array_equal(found.cpu().numpy(), ef)
    assert np.array_equal(out.cpu().numpy().astype(np.int64), np.where(ef == 1, ev, -1))


def test_full_size_1024_maps(F):
    """1024 maps, n log-uniform in [16, 2^20] (about 10^8 keys), 2^24 batched
    lookups at 75 % hits: every lookup against the workload's truth, and the
    tables of a sample of maps (the smallest, the largest and 14 others)
    against the oracle."""
    import torch
    b = W.batched_workload(1024, 16, 1 << 20, 1 << 24, 0.75, seed=4)
    S = F.fks_build_batched(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, b.seeds, dev(b.vals))
    assert (S.status == 0).all()
    out, found = batched_lookup(F, S, b.q_map, b.q_keys)
    assert np.array_equal(found, b.expect_found)
    assert np.array_equal(out, np.where(b.expect_found == 1, b.expect_vals, -1))
    sizes = np.diff(b.seg_offs)
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes))} | set(range(0, 1024, 73))
    for j in sorted(pick):
        k = b.keys[b.seg_offs[j]:b.seg_offs[j + 1]]
        om = O.build_u64(k, b.vals[b.seg_offs[j]:b.seg_offs[j + 1]], seed=int(b.seeds[j]))
        d, s = export(F, S.get(j))
        assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots), j
    del S
    torch.cuda.empty_cache()


def test_more_maps_than_the_shared_segment_table(F):
    """3000 maps (the grouping keeps at most 2048 segment offsets in shared
    memory; beyond that it searches them in global memory), over 2^20 keys in
    all (two radix levels): sampled maps against the oracle, every lookup
    against the workload's truth."""
    import torch
    b = W.batched_workload(3000, 100, 2000, 1 << 18, 0.75, seed=77)
    assert b.seg_offs[-1] >= (1 << 20)
    S = F.fks_build_batched(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, b.seeds, dev(b.vals))
    assert (S.status == 0).all() and len(S) == 3000
    for j in (0, 1, 1499, 2047, 2048, 2999):
        k = b.keys[b.seg_offs[j]:b.seg_offs[j + 1]]
        om = O.build_u64(k, b.vals[b.seg_offs[j]:b.seg_offs[j + 1]], seed=int(b.seeds[j]))
        d, s = export(F, S.get(j))
        assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots), j
    out, found = batched_lookup(F, S, b.q_map, b.q_keys)
    assert np.array_equal(found, b.expect_found)
    assert np.array_equal(out, np.where(b.expect_found == 1, b.expect_vals, -1))
    del S
    torch.cuda.empty_cache()
