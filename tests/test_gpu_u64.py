"""Parity of the device build and lookup over uint64 keys with the CPU oracle.

Bit-exact: descriptors, slot tables and lookup results are integers, so the
device tables must equal the oracle's byte for byte and every lookup output
must match (Sec. 2.2 construction and membership test; Sec. 3.2 lookup).
"""
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


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def u64(a):
    import torch
    return dev(np.ascontiguousarray(a, np.uint64).view(np.int64))


def gpu_build(F, keys, vals, seed, **opts):
    o = F.make_opts(**opts) if opts else None
    return F.fks_build_u64(u64(keys), dev(vals), seed, o)


def gpu_lookup(F, m, q, i64=True, absent=-1):
    import torch
    qt = u64(q)
    out = torch.empty(len(q), dtype=torch.int64 if i64 else torch.int32, device="cuda")
    found = torch.empty(len(q), dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(m, qt, out, found, absent)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int64), found.cpu().numpy()


def assert_same_tables(F, gm, om):
    desc, slots, _ = F.fks_map_export(gm)
    info = F.fks_map_info(gm)
    assert info.round == om.round
    assert info.slots == om.S
    assert np.array_equal(desc, om.desc)
    assert np.array_equal(slots, om.slots)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 1023, 1024, 1025, 5000, (1 << 16) + 7, 300001,
                               (1 << 20) + 12345])
def test_tables_and_lookups_bit_exact(F, n):
    w = W.u64_workload(n, 2 * n + 3, 0.5, seed=n)
    om = O.build_u64(w.keys, w.vals, seed=1234 + n)
    assert om.status == O.OK
    gm = gpu_build(F, w.keys, w.vals, 1234 + n)
    assert_same_tables(F, gm, om)
    out, found = gpu_lookup(F, gm, w.queries, absent=-5)
    oo, of = O.lookup_u64(om, w.queries, absent=-5)
    assert np.array_equal(found, of) and np.array_equal(out, oo)
    assert np.array_equal(found, w.expect_found)


def test_2e16_keys_half_hits_workload(F):
    """2^16 keys, 2^16 queries with 50 % members."""
    w = W.u64_workload(1 << 16, 1 << 16, 0.5, seed=1)
    om = O.build_u64(w.keys, w.vals, seed=1)
    gm = gpu_build(F, w.keys, w.vals, 1)
    assert_same_tables(F, gm, om)
    out, found = gpu_lookup(F, gm, w.queries)
    oo, of = O.lookup_u64(om, w.queries)
    assert np.array_equal(out, oo) and np.array_equal(found, of)


def test_int32_values_and_sentinel(F):
    import torch
    n = 4000
    w = W.u64_workload(n, 3 * n, 0.5, seed=5)
    vals = (np.arange(n, dtype=np.int64) * 7919 - 2**30).astype(np.int32)
    om = O.build_u64(w.keys, vals.astype(np.int64), seed=9)
    gm = F.fks_build_u64(u64(w.keys), dev(vals), 9)
    assert_same_tables(F, gm, om)
    out, found = gpu_lookup(F, gm, w.queries, i64=False, absent=-2**31)
    oo, of = O.lookup_u64(om, w.queries, absent=-2**31)
    assert np.array_equal(out, oo) and np.array_equal(found, of)
    with pytest.raises(F.FksError):
        qt = u64(w.queries)
        F.fks_lookup_u64(gm, qt, torch.empty(len(w.queries), dtype=torch.int32, device="cuda"),
                         None, absent=2**40)


def test_lookup_edge_shapes(F):
    import torch
    n = 3000
    w = W.u64_workload(n, 1001, 0.5, seed=6)
    om = O.build_u64(w.keys, w.vals, seed=3)
    gm = gpu_build(F, w.keys, w.vals, 3)
    # empty batch is a no-op
    F.fks_lookup_u64(gm, u64(np.zeros(0, np.uint64)), None, None)
    # unaligned needles / outputs (scalar path), ragged length
    qt = u64(np.concatenate([np.zeros(1, np.uint64), w.queries]))[1:]
    out = torch.empty(len(w.queries) + 1, dtype=torch.int64, device="cuda")[1:]
    found = torch.empty(len(w.queries) + 3, dtype=torch.uint8, device="cuda")[3:]
    F.fks_lookup_u64(gm, qt, out, found, -1)
    torch.cuda.synchronize()
    oo, of = O.lookup_u64(om, w.queries)
    assert np.array_equal(out.cpu().numpy(), oo) and np.array_equal(found.cpu().numpy(), of)
    # membership only (Sec. 4: membership differs from lookup in not reading the value)
    found2 = torch.empty(len(w.queries), dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(gm, u64(w.queries), None, found2)
    torch.cuda.synchronize()
    assert np.array_equal(found2.cpu().numpy(), of)


def test_duplicates_rejected(F):
    keys = W.key_stream(9, 5000)
    keys[4000] = keys[17]
    with pytest.raises(F.FksError) as e:
        gpu_build(F, keys, np.arange(5000), 1)
    assert e.value.status == F.FKS_ERR_DUPLICATE_KEY
    assert O.build_u64(keys, np.arange(5000), seed=1).status == O.DUPLICATE_KEY
    for n in (2, 100, 5000):
        with pytest.raises(F.FksError) as e:
            gpu_build(F, np.full(n, 42, np.uint64), np.arange(n), 1)
        assert e.value.status == F.FKS_ERR_DUPLICATE_KEY
    # the all-ones key is also handled by the global duplicate test
    with pytest.raises(F.FksError) as e:
        gpu_build(F, np.full(50, 2**64 - 1, np.uint64), np.arange(50), 1)
    assert e.value.status == F.FKS_ERR_DUPLICATE_KEY


def test_forced_reseed_parity(F):
    """bound 1 admits only all-singleton bucket layouts: many level-one rounds;
    the device agrees with the oracle on the outcome and on the table."""
    status_map = {O.BUILD_FAILED: F.FKS_ERR_BUILD_FAILED, O.DUPLICATE_KEY: F.FKS_ERR_DUPLICATE_KEY}
    for n in (5, 7):
        for seed in range(6):
            keys = W.key_stream(40 + seed, n)
            om = O.build_u64(keys, np.arange(n), seed=seed, bound_factor=1, round_cap=400)
            if om.status == O.OK:
                gm = gpu_build(F, keys, np.arange(n), seed, bound_factor=1, round_cap=400)
                assert_same_tables(F, gm, om)
            else:
                with pytest.raises(F.FksError) as e:
                    gpu_build(F, keys, np.arange(n), seed, bound_factor=1, round_cap=400)
                assert e.value.status == status_map[om.status]
    keys = W.key_stream(4, 400)
    assert O.build_u64(keys, np.arange(400), seed=2, bound_factor=1, round_cap=3).status == O.BUILD_FAILED
    with pytest.raises(F.FksError) as e:
        gpu_build(F, keys, np.arange(400), 2, bound_factor=1, round_cap=3)
    assert e.value.status == F.FKS_ERR_BUILD_FAILED


@pytest.mark.parametrize("reject", [3, 70])
def test_forced_level_two_retries_parity(F, reject):
    keys = W.key_stream(6, 20000)
    om = O.build_u64(keys, np.arange(20000), seed=8, reject_attempts=reject)
    gm = gpu_build(F, keys, np.arange(20000), 8, reject_attempts=reject)
    assert_same_tables(F, gm, om)


def test_attempt_cap_exhaustion_parity(F):
    keys = W.key_stream(6, 300)
    with pytest.raises(F.FksError) as e:
        gpu_build(F, keys, np.arange(300), 8, reject_attempts=10, attempt_cap=10, round_cap=4)
    assert e.value.status == F.FKS_ERR_BUILD_FAILED


def crafted_crowded_keys(seed, n_total, crowd):
    """Keys of which `crowd` fall into level-one buckets 0..1023 in round 0
    (more than one partition's shared-memory capacity)."""
    c1 = [np.uint64(x) for x in O.derive(seed, 0, O.TAG_L1, 0)]
    base = W.key_stream(77, n_total)
    cand = W.key_stream(78, int(crowd * n_total / 1024 * 1.3) + 1000)
    with np.errstate(over="ignore"):
        h = (c1[0] * (cand & np.uint64(0xFFFFFFFF)) + c1[1] * (cand >> np.uint64(32)) + c1[2]) >> np.uint64(32)
        b = (h * np.uint64(n_total)) >> np.uint64(32)
    sel = cand[b < 1024][:crowd]
    assert sel.size == crowd
    keys = np.concatenate([sel, base[: n_total - crowd]])
    assert np.unique(keys).size == keys.size
    return keys


def test_overflow_partition_parity(F):
    n, seed = 200000, 31
    keys = crafted_crowded_keys(seed, n, 3000)
    om = O.build_u64(keys, np.arange(n), seed=seed)
    assert om.status == O.OK and om.round == 0
    gm = gpu_build(F, keys, np.arange(n), seed)
    assert F.fks_map_info(gm).overflow_partitions >= 1
    assert_same_tables(F, gm, om)
    q = np.concatenate([keys[::3], W.key_stream(999, 5000)])
    out, found = gpu_lookup(F, gm, q)
    oo, of = O.lookup_u64(om, q)
    assert np.array_equal(out, oo) and np.array_equal(found, of)


def test_overflow_partition_two_level_grouping(F):
    """An oversized partition in a build large enough for the two-level grouping."""
    n, seed = (1 << 20) + 100, 33
    keys = crafted_crowded_keys(seed, n, 2600)
    om = O.build_u64(keys, np.arange(n), seed=seed)
    assert om.status == O.OK and om.round == 0
    gm = gpu_build(F, keys, np.arange(n), seed)
    assert F.fks_map_info(gm).overflow_partitions >= 1
    assert_same_tables(F, gm, om)


def test_deterministic_tables(F):
    w = W.u64_workload(100000, 10, 0.5, seed=12)
    first = None
    for _ in range(5):
        gm = gpu_build(F, w.keys, w.vals, 77)
        desc, slots, _ = F.fks_map_export(gm)
        if first is None:
            first = (desc, slots)
        else:
            assert np.array_equal(first[0], desc) and np.array_equal(first[1], slots)


def test_bounded_wait_times_out_and_context_survives(F):
    w = W.u64_workload(50000, 10, 0.5, seed=13)
    F.fks_test_hold_first_partition(True)
    try:
        with pytest.raises(F.FksError) as e:
            gpu_build(F, w.keys, w.vals, 1, spin_limit=2000)
        assert e.value.status == F.FKS_ERR_TIMEOUT
    finally:
        F.fks_test_hold_first_partition(False)
    om = O.build_u64(w.keys, w.vals, seed=1)
    gm = gpu_build(F, w.keys, w.vals, 1)
    assert_same_tables(F, gm, om)


def test_invalid_arguments(F):
    import torch
    with pytest.raises(F.FksError) as e:
        F.fks_build_u64(u64(np.zeros(0, np.uint64)), dev(np.zeros(0, np.int64)), 1)
    assert e.value.status == F.FKS_ERR_INVALID_ARG
    with pytest.raises(TypeError):
        F.fks_build_u64(u64(np.arange(5, dtype=np.uint64)), dev(np.zeros(5, np.float32)), 1)
    with pytest.raises(F.FksError):
        F.fks_build_u64(u64(np.arange(5, dtype=np.uint64)), dev(np.arange(5)), 1,
                        F.make_opts(bound_factor=65))


@pytest.mark.parametrize("kind", W.STRUCTURED_KINDS)
def test_structured_key_sets_bit_exact(F, kind):
    """Consecutive integers, keys equal in one or both 32-bit halves, single
    bits and complements, the top of the range: tables and lookups equal the
    oracle's."""
    keys = W.structured_keys(kind, 5000)
    vals = np.arange(keys.size, dtype=np.int64) * 3 - 5
    om = O.build_u64(keys, vals, seed=23)
    assert om.status == O.OK
    gm = gpu_build(F, keys, vals, 23)
    assert_same_tables(F, gm, om)
    q = np.concatenate([keys, np.setdiff1d(W.structured_keys(kind, 9000), keys)[:2000]])
    out, found = gpu_lookup(F, gm, q)
    oo, of = O.lookup_u64(om, q)
    assert np.array_equal(out, oo) and np.array_equal(found, of)


def test_binding_refuses_mismatched_buffers(F):
    """Buffers the C ABI would misread are refused by the binding before any
    launch: 32-bit keys, an int64 result buffer for an int32 map, a strided
    needle view, a short flag buffer.  The map answers correctly afterwards."""
    import torch
    n = 2000
    w = W.u64_workload(n, 500, 0.5, seed=21)
    vals = np.arange(n, dtype=np.int32)
    with pytest.raises(TypeError, match="keys"):
        F.fks_build_u64(dev(w.keys.astype(np.int32)), dev(vals), 4)
    gm = F.fks_build_u64(u64(w.keys), dev(vals), 4)
    qt = u64(w.queries)
    with pytest.raises(TypeError, match="out_vals"):
        F.fks_lookup_u64(gm, qt, torch.empty(500, dtype=torch.int64, device="cuda"), None)
    with pytest.raises(ValueError, match="contiguous"):
        F.fks_lookup_u64(gm, u64(np.repeat(w.queries, 2))[::2], None,
                         torch.empty(500, dtype=torch.uint8, device="cuda"))
    with pytest.raises(ValueError, match="out_found"):
        F.fks_lookup_u64(gm, qt, None, torch.empty(499, dtype=torch.uint8, device="cuda"))
    out, found = gpu_lookup(F, gm, w.queries, i64=False)
    om = O.build_u64(w.keys, vals.astype(np.int64), seed=4)
    oo, of = O.lookup_u64(om, w.queries)
    assert np.array_equal(out, oo) and np.array_equal(found, of)


def test_full_size_2e26_keys_bit_exact(F):
    """2^26 keys, 2^26 queries at 90 % hits, the benchmark's launch
    configuration: whole tables and every lookup output against the oracle."""
    import torch
    n = 1 << 26
    w = W.u64_workload(n, n, 0.9, seed=2)
    gm = gpu_build(F, w.keys, w.vals, 2)
    out, found = gpu_lookup(F, gm, w.queries)
    assert np.array_equal(found, w.expect_found)
    assert np.array_equal(out, np.where(w.expect_found == 1, w.expect_vals, -1))
    om = O.build_u64(w.keys, w.vals, seed=2)
    assert_same_tables(F, gm, om)
    oo, of = O.lookup_u64(om, w.queries)
    assert np.array_equal(out, oo) and np.array_equal(found, of)
    del gm
    torch.cuda.empty_cache()
