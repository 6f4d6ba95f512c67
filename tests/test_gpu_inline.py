"""Inline-singleton records (build option inline_singletons): the records the
device writes equal the oracle's, written out from the oracle's own table,
and the record-first lookups answer exactly as the oracle's two-probe lookup,
on random, structured and crafted key sets, in level-one rounds after the
first, through the partition overflow path, with int32 values."""
import numpy as np
import pytest

import oracle as O
from paper_2508_11443_b300 import workloads as W
from test_gpu_u64 import crafted_crowded_keys

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


def check(F, keys, vals, seed, queries, **opts):
    import torch
    om = O.build_u64(keys, vals.astype(np.int64), seed=seed, **{k: v for k, v in opts.items() if k != "inline_singletons"})
    assert om.status == O.OK
    gm = F.fks_build_u64(dev(keys), dev(vals), seed, F.make_opts(inline_singletons=1, **opts))
    info = F.fks_map_info(gm)
    assert info.inline_singletons == 1 and info.round == om.round
    d, s, _ = F.fks_map_export(gm)
    assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots)  # the paper's tables, unchanged
    assert np.array_equal(F.fks_map_export_records(gm), O.inline_records(om))
    i64 = vals.dtype == np.int64
    out = torch.empty(len(queries), dtype=torch.int64 if i64 else torch.int32, device="cuda")
    found = torch.empty(len(queries), dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(gm, dev(queries), out, found, -1)
    torch.cuda.synchronize()
    oo, of = O.lookup_u64(om, queries)
    assert np.array_equal(found.cpu().numpy(), of)
    assert np.array_equal(out.cpu().numpy().astype(np.int64), oo)
    return om, gm


@pytest.mark.parametrize("n", [1, 2, 3, 1000, (1 << 16) + 3, (1 << 20) + 7])
def test_records_and_lookups(F, n):
    w = W.u64_workload(n, 2 * n + 5, 0.5, seed=n + 90)
    check(F, w.keys, w.vals, 91, w.queries)


@pytest.mark.parametrize("kind", W.STRUCTURED_KINDS)
def test_structured_keys(F, kind):
    keys = W.structured_keys(kind, 5000)
    extra = np.array([0, 1, 2**63, 2**64 - 1], np.uint64)
    q = np.concatenate([keys, np.setdiff1d(W.structured_keys(kind, 9000), keys)[:2000], extra])
    check(F, keys, np.arange(keys.size, dtype=np.int64) * 3 - 5, 92, q)


def test_int32_values_later_round_and_unaligned(F):
    """int32 values (sign-extended in the record), a table from level-one round
    >= 1, and needles / results at unaligned addresses (the scalar path)."""
    import torch
    keys = W.key_stream(81, 3000)
    for seed in range(200):
        om = O.build_u64(keys, np.arange(3000), seed=seed, bound_factor=2)
        if om.status == O.OK and om.round >= 1:
            break
    assert om.round >= 1
    vals = (np.arange(3000, dtype=np.int64) * 7919 - 2**30).astype(np.int32)
    q = np.concatenate([keys, W.key_stream(82, 1001)])
    _, gm = check(F, keys, vals, seed, q, bound_factor=2)
    qt = dev(np.concatenate([np.zeros(1, np.uint64), q]))[1:]
    out = torch.empty(q.size + 1, dtype=torch.int32, device="cuda")[1:]
    found = torch.empty(q.size + 3, dtype=torch.uint8, device="cuda")[3:]
    F.fks_lookup_u64(gm, qt, out, found, -7)
    torch.cuda.synchronize()
    om32 = O.build_u64(keys, vals.astype(np.int64), seed=seed, bound_factor=2)
    oo, of = O.lookup_u64(om32, q, absent=-7)
    assert np.array_equal(found.cpu().numpy(), of) and np.array_equal(out.cpu().numpy().astype(np.int64), oo)


def test_overflow_partition(F):
    """Records of buckets in a partition above the shared-memory capacity,
    written by the overflow kernel."""
    n, seed = 200000, 31
    keys = crafted_crowded_keys(seed, n, 3000)
    q = np.concatenate([keys[::3], W.key_stream(999, 5000)])
    _, gm = check(F, keys, np.arange(n, dtype=np.int64), seed, q)
    assert F.fks_map_info(gm).overflow_partitions >= 1


def test_refused_where_it_does_not_apply(F):
    keys = W.key_stream(5, 100)
    vals = np.arange(100, dtype=np.int64)
    for bad in (dict(inline_singletons=1, keys_per_bucket=2), dict(inline_singletons=2)):
        with pytest.raises(F.FksError) as e:
            F.fks_build_u64(dev(keys), dev(vals), 1, F.make_opts(**bad))
        assert e.value.status == F.FKS_ERR_INVALID_ARG
    s = W.string_workload(100, 1, 1.0, seed=6)
    with pytest.raises(F.FksError) as e:
        F.fks_build_bytes(dev(s.ctx), dev(s.offs), dev(s.vals), 1, F.make_opts(inline_singletons=1))
    assert e.value.status == F.FKS_ERR_INVALID_ARG
    with pytest.raises(F.FksError) as e:
        F.fks_build_batched(F.FKS_KEY_U64, dev(keys), None, None, np.array([0, 50, 100]), np.array([1, 2]),
                            dev(vals), F.make_opts(inline_singletons=1))
    assert e.value.status == F.FKS_ERR_INVALID_ARG
    plain = F.fks_build_u64(dev(keys), dev(vals), 1)
    assert F.fks_map_info(plain).inline_singletons == 0
    with pytest.raises(F.FksError):
        F.fks_map_export_records(plain)


def test_checkpoint_of_a_map_with_records(F, tmp_path):
    """A checkpoint holds the paper's tables only: the imported map has no
    records and answers through its descriptors, with the same results."""
    import torch
    w = W.u64_workload(30000, 40000, 0.5, seed=95)
    om, gm = check(F, w.keys, w.vals, 96, w.queries)
    path = str(tmp_path / "inline_map.npz")
    F.fks_map_save(gm, path)
    back = F.fks_map_load(path)
    assert F.fks_map_info(back).inline_singletons == 0
    out = torch.empty(len(w.queries), dtype=torch.int64, device="cuda")
    found = torch.empty(len(w.queries), dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(back, dev(w.queries), out, found, -1)
    torch.cuda.synchronize()
    oo, of = O.lookup_u64(om, w.queries)
    assert np.array_equal(found.cpu().numpy(), of) and np.array_equal(out.cpu().numpy(), oo)
