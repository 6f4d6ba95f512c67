"""Launch shapes and the autotuner on the GPU: every shape builds the same
tables (byte for byte against the oracle) and answers every lookup the same;
fks_autotune picks candidates from the documented sets and later builds use
them, still bit-exact."""
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
    fks.fks_tuning_reset()
    yield fks
    fks.fks_tuning_reset()


def dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


SHAPES = [dict(thread_search_max=1), dict(thread_search_max=2), dict(part_ctas_per_sm=1), dict(part_prefetch=0),
          dict(part_prefetch=1, thread_search_max=3),
          dict(split_min_keys_log2=16), dict(split_min_keys_log2=30, scatter_blocks_per_sm=3),
          dict(thread_search_max=1, part_ctas_per_sm=1, split_min_keys_log2=12, scatter_blocks_per_sm=32)]


def install(F, kind, lam, **fields):
    t = F.fks_tuning_get(kind, lam)
    for k, v in fields.items():
        setattr(t, k, v)
    F.fks_tuning_set(t)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("lam", [1, 8])
def test_build_shapes_give_the_same_tables(F, shape, lam):
    n = (1 << 17) + 12345  # several partitions and a ragged last one
    w = W.u64_workload(n, 4096, 0.5, seed=7)
    om = O.build_u64(w.keys, w.vals, seed=5, keys_per_bucket=lam)
    F.fks_tuning_reset()
    install(F, F.FKS_KEY_U64, lam, **shape)
    m = F.fks_build_u64(dev(w.keys), dev(w.vals), 5, opts=F.make_opts(keys_per_bucket=lam))
    d, s, _ = F.fks_map_export(m)
    assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots)
    F.fks_tuning_reset()


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[3], SHAPES[5], SHAPES[7]])
def test_string_build_shapes_give_the_same_tables(F, shape):
    s = W.string_workload(70000, 100, 0.5, seed=8)
    om = O.build_bytes(s.ctx, s.offs, s.vals, seed=9)
    install(F, F.FKS_KEY_BYTES, 1, **shape)
    m = F.fks_build_bytes(dev(s.ctx), dev(s.offs), dev(s.vals.astype(np.int32)), 9)
    d, sl, _ = F.fks_map_export(m)
    assert np.array_equal(d, om.desc) and np.array_equal(sl, om.slots)
    F.fks_tuning_reset()


@pytest.mark.parametrize("qpt", [2, 4, 8])
@pytest.mark.parametrize("block", [128, 512])
@pytest.mark.parametrize("per_sm", [1, 16])
def test_lookup_shapes_give_the_same_answers(F, qpt, block, per_sm):
    import torch
    w = W.u64_workload(50000, 30011, 0.6, seed=11)  # odd needle count: a ragged tail
    m = F.fks_build_u64(dev(w.keys), dev(w.vals), 3)
    install(F, F.FKS_KEY_U64, 1, lookup_queries_per_thread=qpt, lookup_block=block, lookup_blocks_per_sm=per_sm)
    exp_v = np.where(w.expect_found == 1, w.expect_vals, -1)
    for i64 in (True, False):
        for shift in (0, 1):  # shift 1: unaligned buffers take the scalar path
            q = dev(np.concatenate([np.zeros(shift, np.uint64), w.queries]))[shift:]
            out = torch.empty(len(w.queries) + shift, dtype=torch.int64 if i64 else torch.int32,
                              device="cuda")[shift:]
            found = torch.empty(len(w.queries) + shift, dtype=torch.uint8, device="cuda")[shift:]
            if not i64:
                m32 = F.fks_build_u64(dev(w.keys), dev(w.vals.astype(np.int32)), 3)
                F.fks_lookup_u64(m32, q, out, found, -1)
            else:
                F.fks_lookup_u64(m, q, out, found, -1)
            torch.cuda.synchronize()
            assert np.array_equal(found.cpu().numpy(), w.expect_found)
            assert np.array_equal(out.cpu().numpy().astype(np.int64), exp_v)
    F.fks_tuning_reset()


def test_autotune_u64_then_build_bit_exact(F):
    F.fks_tuning_reset()
    t, rows = F.fks_autotune(F.FKS_KEY_U64, 1, n=1 << 20, nq=1 << 20, seed=3)
    assert t.tuned == 1 and t.sample_keys == 1 << 20 and t.build_ms > 0 and t.lookup_ms > 0
    assert t.thread_search_max in (1, 2, 3) and t.part_ctas_per_sm in (0, 1, 2)
    assert t.lookup_queries_per_thread in (2, 4, 8) and t.lookup_block in (128, 256, 512)
    assert t.lookup_blocks_per_sm in (4, 8, 32, 128, 1024)
    assert t.part_prefetch in (0, 1)
    assert len(rows) >= 3 + 2 + 2 + 2 + 9 + 5 and all(ms > 0 for _, _, ms in rows)
    got = F.fks_tuning_get(F.FKS_KEY_U64, 1)
    assert got.as_dict() == t.as_dict()
    # builds and lookups now run at the tuned shape, with the same results
    w = W.u64_workload((1 << 18) + 77, 5000, 0.5, seed=12)
    om = O.build_u64(w.keys, w.vals, seed=2)
    m = F.fks_build_u64(dev(w.keys), dev(w.vals), 2)
    d, s, _ = F.fks_map_export(m)
    assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots)
    import torch
    out = torch.empty(5000, dtype=torch.int64, device="cuda")
    found = torch.empty(5000, dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(m, dev(w.queries), out, found, -1)
    torch.cuda.synchronize()
    assert np.array_equal(found.cpu().numpy(), w.expect_found)
    F.fks_tuning_reset()


def test_autotune_strings(F):
    t, rows = F.fks_autotune(F.FKS_KEY_BYTES, 1, n=1 << 16, seed=4)
    assert t.tuned == 1 and t.key_kind == F.FKS_KEY_BYTES and t.build_ms > 0
    assert all(p not in ("lookup_blocks_per_sm",) for p, _, _ in rows)
    s = W.string_workload(20000, 100, 0.5, seed=13)
    om = O.build_bytes(s.ctx, s.offs, s.vals, seed=6)
    m = F.fks_build_bytes(dev(s.ctx), dev(s.offs), dev(s.vals), 6)
    d, sl, _ = F.fks_map_export(m)
    assert np.array_equal(d, om.desc) and np.array_equal(sl, om.slots)
    F.fks_tuning_reset()


@pytest.mark.parametrize("lam,fields", [
    (1, dict(lookup_queries_per_thread=4, lookup_block=512, lookup_blocks_per_sm=1024)),
    (16, dict(thread_search_max=2, part_prefetch=0, lookup_queries_per_thread=4, lookup_block=256,
              lookup_blocks_per_sm=1024))])
def test_full_size_at_the_benchmark_shapes(F, lam, fields):
    """2^26 keys and 2^26 queries (90 % hits) at the launch shapes the
    benchmark's autotuner chose on a B300: every lookup output against the
    workload's truth, and the tables equal to a build at the default shapes
    (whose tables the full-size oracle tests pin)."""
    import torch
    n = 1 << 26
    w = W.u64_workload(n, n, 0.9, seed=2)
    keys, vals, q = dev(w.keys), dev(w.vals), dev(w.queries)
    o = F.make_opts(keys_per_bucket=lam)
    F.fks_tuning_reset()
    ref = F.fks_build_u64(keys, vals, 2, o)
    d0, s0, _ = F.fks_map_export(ref)
    del ref
    install(F, F.FKS_KEY_U64, lam, **fields)
    m = F.fks_build_u64(keys, vals, 2, o)
    d1, s1, _ = F.fks_map_export(m)
    assert np.array_equal(d0, d1) and np.array_equal(s0, s1)
    del d0, s0, d1, s1
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    found = torch.empty(n, dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(m, q, out, found, -1)
    torch.cuda.synchronize()
    assert np.array_equal(found.cpu().numpy(), w.expect_found)
    assert np.array_equal(out.cpu().numpy(), np.where(w.expect_found == 1, w.expect_vals, -1))
    F.fks_tuning_reset()
    del m, out, found, keys, vals, q
    torch.cuda.empty_cache()
