"""Checkpoint / resume of built maps: fks_map_export -> a file -> fks_map_import
gives a map with the same tables and the same answers (and the oracle's);
descriptors that do not match the metadata are rejected before any upload."""
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


def lookup(F, m, q, i64=True):
    import torch
    out = torch.empty(len(q), dtype=torch.int64 if i64 else torch.int32, device="cuda")
    found = torch.empty(len(q), dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(m, dev(q), out, found, -1)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int64), found.cpu().numpy()


@pytest.mark.parametrize("lam,i64", [(1, True), (4, False), (16, True)])
def test_u64_map_survives_save_and_load(F, tmp_path, lam, i64):
    w = W.u64_workload(100003, 20000, 0.5, seed=lam)
    vals = w.vals if i64 else w.vals.astype(np.int32)
    m = F.fks_build_u64(dev(w.keys), dev(vals), 77, opts=F.make_opts(keys_per_bucket=lam))
    path = str(tmp_path / "map.npz")
    F.fks_map_save(m, path)
    r = F.fks_map_load(path)
    d1, s1, _ = F.fks_map_export(m)
    d2, s2, _ = F.fks_map_export(r)
    assert np.array_equal(d1, d2) and np.array_equal(s1, s2)
    om = O.build_u64(w.keys, w.vals, seed=77, keys_per_bucket=lam)
    assert np.array_equal(d2, om.desc) and np.array_equal(s2, om.slots)
    a, b = F.fks_map_info(m), F.fks_map_info(r)
    for k in ("n", "seed", "round", "slots", "slot_capacity", "buckets", "keys_per_bucket", "val_type"):
        assert getattr(a, k) == getattr(b, k), k
    out, found = lookup(F, r, w.queries, i64)
    assert np.array_equal(found, w.expect_found)
    assert np.array_equal(out, np.where(w.expect_found == 1, w.expect_vals, -1))


def test_string_map_survives_save_and_load(F, tmp_path):
    import torch
    s = W.string_workload(30000, 8000, 0.5, seed=21)
    m = F.fks_build_bytes(dev(s.ctx), dev(s.offs), dev(s.vals.astype(np.int32)), 5)
    path = str(tmp_path / "smap.npz")
    F.fks_map_save(m, path)
    del m
    r = F.fks_map_load(path)
    out = torch.empty(8000, dtype=torch.int32, device="cuda")
    found = torch.empty(8000, dtype=torch.uint8, device="cuda")
    F.fks_lookup_bytes(r, dev(s.qctx), dev(s.qoffs), out, found, -1)
    torch.cuda.synchronize()
    assert np.array_equal(found.cpu().numpy(), s.expect_found)
    assert np.array_equal(out.cpu().numpy().astype(np.int64), np.where(s.expect_found == 1, s.expect_vals, -1))
    om = O.build_bytes(s.ctx, s.offs, s.vals, seed=5)
    d, sl, ctx = F.fks_map_export(r)
    assert np.array_equal(d, om.desc) and np.array_equal(sl, om.slots) and np.array_equal(ctx, s.ctx)


def test_a_map_of_a_batched_set_can_be_saved(F, tmp_path):
    b = W.batched_workload(5, 100, 5000, 1000, 0.75, seed=2)
    S = F.fks_build_batched(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, b.seeds, dev(b.vals))
    path = str(tmp_path / "m3.npz")
    F.fks_map_save(S.get(3), path)
    r = F.fks_map_load(path)
    k = b.keys[b.seg_offs[3]:b.seg_offs[4]]
    out, found = lookup(F, r, k)
    assert found.all() and np.array_equal(out, b.vals[b.seg_offs[3]:b.seg_offs[4]])


def test_inconsistent_tables_are_rejected(F):
    w = W.u64_workload(5000, 10, 0.5, seed=3)
    m = F.fks_build_u64(dev(w.keys), dev(w.vals), 1)
    info = F.fks_map_info(m)
    desc, slots, _ = F.fks_map_export(m)
    bad = desc.copy()
    nz = np.nonzero((bad >> np.uint64(32)) & np.uint64(0xFFFFF))[0]
    bad[nz[5]] += np.uint64(1)  # a bucket's slot range moved by one
    with pytest.raises(F.FksError) as e:
        F.fks_map_import(info, bad, slots)
    assert e.value.status == F.FKS_ERR_INVALID_ARG
    info.n += 1  # the key count no longer matches the descriptors
    with pytest.raises(F.FksError):
        F.fks_map_import(info, desc, slots)
