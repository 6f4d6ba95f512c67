"""Parity of the bucket-count variant (nb = ceil(n / lambda) level-one buckets)
with the CPU oracle: descriptors, slot tables and lookup outputs bit-exact,
for uint64 and string keys, per-call and batched builds, the shared-memory,
direct-write and global-memory (overflow) partition paths, and the full
2^26-key size in the benchmark's launch configuration."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2508_11443_b300 import workloads as W

pytestmark = pytest.mark.gpu

LAMBDAS = [2, 4, 8, 16]
LOG_B = {1: 10, 2: 9, 4: 8, 8: 7, 16: 6}   # buckets per partition of the device build


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


def gpu_lookup(F, m, q, absent=-1):
    import torch
    out = torch.empty(len(q), dtype=torch.int64, device="cuda")
    found = torch.empty(len(q), dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(m, dev(np.asarray(q, np.uint64)), out, found, absent)
    torch.cuda.synchronize()
    return out.cpu().numpy(), found.cpu().numpy()


def same_tables(F, gm, om):
    desc, slots, _ = F.fks_map_export(gm)
    info = F.fks_map_info(gm)
    assert info.round == om.round and info.slots == om.S
    assert info.buckets == om.nb == desc.size
    assert info.keys_per_bucket == om.keys_per_bucket
    assert np.array_equal(desc, om.desc)
    assert np.array_equal(slots, om.slots)


@pytest.mark.parametrize("lam", LAMBDAS)
@pytest.mark.parametrize("n", [1, 3, 17, 1000, 1025, 4099, (1 << 16) + 7, 300001, (1 << 20) + 12345])
def test_tables_and_lookups_bit_exact(F, lam, n):
    w = W.u64_workload(n, 2 * n + 3, 0.5, seed=n + lam)
    om = O.build_u64(w.keys, w.vals, seed=99 + n, keys_per_bucket=lam)
    assert om.status == O.OK
    gm = F.fks_build_u64(dev(w.keys), dev(w.vals), 99 + n, F.make_opts(keys_per_bucket=lam))
    same_tables(F, gm, om)
    out, found = gpu_lookup(F, gm, w.queries, absent=-5)
    oo, of = O.lookup_u64(om, w.queries, absent=-5)
    assert np.array_equal(found, of) and np.array_equal(out, oo)
    assert np.array_equal(found, w.expect_found)


def test_lambda1_option_equals_default(F):
    w = W.u64_workload(70000, 10, 0.5, seed=3)
    a = F.fks_build_u64(dev(w.keys), dev(w.vals), 5)
    b = F.fks_build_u64(dev(w.keys), dev(w.vals), 5, F.make_opts(keys_per_bucket=1, bound_factor=4))
    da, sa, _ = F.fks_map_export(a)
    db, sb, _ = F.fks_map_export(b)
    assert np.array_equal(da, db) and np.array_equal(sa, sb)


def crowded_keys(seed, n, lam, crowd, first_buckets):
    """n keys of which `crowd` fall, in round 0, into level-one buckets
    0 .. first_buckets - 1 of an nb = ceil(n / lam) bucket map."""
    nb = -(-n // lam)
    c1 = [np.uint64(x) for x in O.derive(seed, 0, O.TAG_L1, 0)]
    cand = W.key_stream(seed + 1000, int(crowd * nb / first_buckets * 1.3) + 4000)
    with np.errstate(over="ignore"):
        h = (c1[0] * (cand & np.uint64(0xFFFFFFFF)) + c1[1] * (cand >> np.uint64(32)) + c1[2]) >> np.uint64(32)
        b = (h * np.uint64(nb)) >> np.uint64(32)
    sel = cand[b < first_buckets][:crowd]
    assert sel.size == crowd
    rest = W.key_stream(seed + 2000, n)
    rest = rest[~np.isin(rest, sel)][: n - crowd]
    keys = np.concatenate([sel, rest])
    assert keys.size == n and np.unique(keys).size == n
    return keys


def check_crafted(F, keys, seed, lam, expect_overflow):
    n = keys.size
    om = O.build_u64(keys, np.arange(n), seed=seed, keys_per_bucket=lam)
    assert om.status == O.OK and om.round == 0
    gm = F.fks_build_u64(dev(keys), dev(np.arange(n)), seed, F.make_opts(keys_per_bucket=lam))
    assert (F.fks_map_info(gm).overflow_partitions >= 1) == expect_overflow
    same_tables(F, gm, om)
    q = np.concatenate([keys[::3], W.key_stream(seed + 3000, 5000)])
    out, found = gpu_lookup(F, gm, q)
    oo, of = O.lookup_u64(om, q)
    assert np.array_equal(out, oo) and np.array_equal(found, of)


def test_large_bucket_direct_write_partition(F):
    """A 200-key bucket (searched by the whole CTA) in a partition whose slot
    image (> 40000 slots) is written straight to global memory."""
    lam, seed, n = 16, 41, 50000
    keys = crowded_keys(seed, n, lam, 200, 1)
    check_crafted(F, keys, seed, lam, expect_overflow=False)


def test_overflow_partition(F):
    """3000 keys in the first partition's 128 buckets (lambda 8): more keys than
    one partition holds in shared memory, built through global memory."""
    lam, seed, n = 8, 43, 200000
    keys = crowded_keys(seed, n, lam, 3000, 1 << LOG_B[lam])
    check_crafted(F, keys, seed, lam, expect_overflow=True)


def test_overflow_partition_two_level_grouping(F):
    lam, seed, n = 4, 45, (1 << 20) + 100
    keys = crowded_keys(seed, n, lam, 2600, 1 << LOG_B[lam])
    check_crafted(F, keys, seed, lam, expect_overflow=True)


@pytest.mark.parametrize("lam", [4, 16])
@pytest.mark.parametrize("n", [1, 5, 3001, 20000])
def test_strings(F, lam, n):
    import torch
    w = W.string_workload(n, 2 * n + 1, 0.5, seed=n + lam)
    om = O.build_bytes(w.ctx, w.offs, w.vals, seed=7 + n, keys_per_bucket=lam)
    assert om.status == O.OK
    ctx = w.ctx if w.ctx.size else np.zeros(1, np.uint8)
    gm = F.fks_build_bytes(dev(ctx), dev(w.offs), dev(w.vals), 7 + n, F.make_opts(keys_per_bucket=lam))
    same_tables(F, gm, om)
    qctx = w.qctx if w.qctx.size else np.zeros(1, np.uint8)
    out = torch.empty(len(w.qoffs) - 1, dtype=torch.int64, device="cuda")
    found = torch.empty(len(w.qoffs) - 1, dtype=torch.uint8, device="cuda")
    F.fks_lookup_bytes(gm, dev(qctx), dev(w.qoffs), out, found, -3)
    torch.cuda.synchronize()
    oo, of = O.lookup_bytes(om, w.qctx, w.qoffs, absent=-3)
    assert np.array_equal(found.cpu().numpy(), of) and np.array_equal(out.cpu().numpy(), oo)


@pytest.mark.parametrize("lam", [2, 8, 16])
def test_batched(F, lam):
    import torch
    b = W.batched_workload(40, 1, 1 << 14, 20000, 0.75, seed=50 + lam)
    S = F.fks_build_batched(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, b.seeds, dev(b.vals),
                            F.make_opts(keys_per_bucket=lam))
    assert (S.status == 0).all()
    for j in range(len(S)):
        k = b.keys[b.seg_offs[j]:b.seg_offs[j + 1]]
        v = b.vals[b.seg_offs[j]:b.seg_offs[j + 1]]
        om = O.build_u64(k, v, seed=int(b.seeds[j]), keys_per_bucket=lam)
        same_tables(F, S.get(j), om)
    out = torch.empty(len(b.q_keys), dtype=torch.int64, device="cuda")
    found = torch.empty(len(b.q_keys), dtype=torch.uint8, device="cuda")
    F.fks_lookup_batched(S, dev(b.q_map.astype(np.uint32)), q=dev(b.q_keys), out_vals=out, out_found=found)
    torch.cuda.synchronize()
    assert np.array_equal(found.cpu().numpy(), b.expect_found)
    assert np.array_equal(out.cpu().numpy(), np.where(b.expect_found == 1, b.expect_vals, -1))


def test_invalid_options(F):
    w = W.u64_workload(1000, 10, 0.5, seed=1)
    for bad in (dict(keys_per_bucket=3), dict(keys_per_bucket=32), dict(bound_factor=65)):
        with pytest.raises(F.FksError) as e:
            F.fks_build_u64(dev(w.keys), dev(w.vals), 1, F.make_opts(**bad))
        assert e.value.status == F.FKS_ERR_INVALID_ARG
    # bound * n beyond the 32-bit slot offsets: rejected before any key is read
    k = dev(w.keys)
    h = ctypes.c_void_p()
    o = F.make_opts(keys_per_bucket=16)
    st = F.lib().fks_build_u64(ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(k.data_ptr()), F.FKS_VAL_I64,
                               1 << 27, 1, ctypes.byref(o), None, None, ctypes.byref(h))
    assert st == F.FKS_ERR_INVALID_ARG and not h.value
    # the allocation-free build takes one bucket per key only
    import torch
    desc = torch.empty(1000, dtype=torch.int64, device="cuda")
    slots = torch.empty(2 * 4 * 1000, dtype=torch.int64, device="cuda")
    with pytest.raises(F.FksError) as e:
        F.fks_build_u64_noalloc(dev(w.keys), dev(w.vals), 1, desc, slots, F.make_opts(keys_per_bucket=2))
    assert e.value.status == F.FKS_ERR_INVALID_ARG


@pytest.mark.parametrize("lam", [8, 16])
def test_full_size_bit_exact(F, lam):
    """2^26 keys, 2^26 queries at 90 % hits: whole tables and every lookup
    output against the oracle."""
    import torch
    n = 1 << 26
    w = W.u64_workload(n, n, 0.9, seed=2)
    gm = F.fks_build_u64(dev(w.keys), dev(w.vals), 2, F.make_opts(keys_per_bucket=lam))
    out, found = gpu_lookup(F, gm, w.queries)
    assert np.array_equal(found, w.expect_found)
    assert np.array_equal(out, np.where(w.expect_found == 1, w.expect_vals, -1))
    om = O.build_u64(w.keys, w.vals, seed=2, keys_per_bucket=lam)
    same_tables(F, gm, om)
    del gm
    torch.cuda.empty_cache()
