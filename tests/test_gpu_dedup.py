"""from_array (opts.dedup = 1): inputs with equal keys, the first occurrence in
input order wins (per map in batched builds).  The device maps must equal,
byte for byte, the oracle's build of the pairs the oracle's first-occurrence
rule keeps (string maps over the kept strings' bytes in input order)."""
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


def same_tables(F, gm, om):
    desc, slots, ctx = F.fks_map_export(gm)
    info = F.fks_map_info(gm)
    assert info.n == om.n and info.round == om.round and info.slots == om.S
    assert np.array_equal(desc, om.desc)
    assert np.array_equal(slots, om.slots)
    return ctx


def dup_keys(u, universe, seed):
    rng = np.random.default_rng(seed)
    base = W.key_stream(seed + 100, universe)
    return base[rng.integers(0, universe, u)]


@pytest.mark.parametrize("u,universe", [(1, 1), (5, 2), (1000, 300), (100000, 20000), ((1 << 21) + 77, 1500000),
                                        (3000, 3000)])
@pytest.mark.parametrize("i64", [True, False])
def test_u64_first_occurrence(F, u, universe, i64):
    import torch
    keys = dup_keys(u, universe, u + universe)
    vals = np.arange(u, dtype=np.int64 if i64 else np.int32) * 3 + 1
    keep = O.dedup_keep(keys=keys).astype(bool)
    om = O.build_u64(keys[keep], vals[keep].astype(np.int64), seed=5)
    assert om.status == O.OK
    gm = F.fks_build_u64(dev(keys), dev(vals), 5, F.make_opts(dedup=1))
    same_tables(F, gm, om)
    q = np.concatenate([keys[: 5000], W.key_stream(7777, 1000)])
    out = torch.empty(q.size, dtype=torch.int64 if i64 else torch.int32, device="cuda")
    found = torch.empty(q.size, dtype=torch.uint8, device="cuda")
    F.fks_lookup_u64(gm, dev(q), out, found, -1)
    torch.cuda.synchronize()
    oo, of = O.lookup_u64(om, q)
    assert np.array_equal(found.cpu().numpy(), of) and np.array_equal(out.cpu().numpy().astype(np.int64), oo)


def test_u64_without_duplicates_equals_nodup(F):
    w = W.u64_workload(50000, 10, 0.5, seed=8)
    a = F.fks_build_u64(dev(w.keys), dev(w.vals), 9)
    b = F.fks_build_u64(dev(w.keys), dev(w.vals), 9, F.make_opts(dedup=1))
    da, sa, _ = F.fks_map_export(a)
    db, sb, _ = F.fks_map_export(b)
    assert np.array_equal(da, db) and np.array_equal(sa, sb)
    # and with duplicates the plain build refuses
    keys = np.concatenate([w.keys, w.keys[:10]])
    with pytest.raises(F.FksError) as e:
        F.fks_build_u64(dev(keys), dev(np.arange(keys.size)), 9)
    assert e.value.status == F.FKS_ERR_DUPLICATE_KEY


def test_all_equal_keys(F):
    keys = np.full(4096, 0xDEADBEEF, np.uint64)
    gm = F.fks_build_u64(dev(keys), dev(np.arange(4096)), 1, F.make_opts(dedup=1, keys_per_bucket=4))
    info = F.fks_map_info(gm)
    assert info.n == 1
    om = O.build_u64(keys[:1], np.arange(1), seed=1, keys_per_bucket=4)
    same_tables(F, gm, om)


def strings_with_dups(u, seed):
    rng = np.random.default_rng(seed)
    pool = W.string_workload(max(8, u // 4), 1, 0.5, seed=seed)
    lens = np.diff(pool.offs)
    pick = rng.integers(0, lens.size, u)
    pieces = [bytes(pool.ctx[pool.offs[i]:pool.offs[i + 1]]) for i in pick]
    pieces[::97] = [b""] * len(pieces[::97])  # some empty strings (equal to each other)
    offs = np.concatenate([[0], np.cumsum([len(p) for p in pieces])]).astype(np.int64)
    ctx = np.frombuffer(b"".join(pieces), np.uint8) if offs[-1] else np.zeros(0, np.uint8)
    return ctx, offs


def compact(ctx, offs, keep):
    pieces = [bytes(ctx[offs[i]:offs[i + 1]]) for i in np.nonzero(keep)[0]]
    noffs = np.concatenate([[0], np.cumsum([len(p) for p in pieces])]).astype(np.int64)
    nctx = np.frombuffer(b"".join(pieces), np.uint8) if noffs[-1] else np.zeros(0, np.uint8)
    return nctx, noffs


@pytest.mark.parametrize("u", [1, 7, 5000, 60000])
def test_strings_first_occurrence(F, u):
    ctx, offs = strings_with_dups(u, u + 3)
    vals = np.arange(u, dtype=np.int64)
    keep = O.dedup_keep(ctx=ctx, offs=offs).astype(bool)
    nctx, noffs = compact(ctx, offs, keep)
    om = O.build_bytes(nctx, noffs, vals[keep], seed=11)
    assert om.status == O.OK
    gctx = ctx if ctx.size else np.zeros(1, np.uint8)
    gm = F.fks_build_bytes(dev(gctx), dev(offs), dev(vals), 11, F.make_opts(dedup=1))
    mctx = same_tables(F, gm, om)
    assert np.array_equal(mctx, nctx)


def test_batched_per_map(F):
    rng = np.random.default_rng(21)
    sizes = rng.integers(1, 3000, 24)
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    shared = W.key_stream(55, 500)
    keys = np.concatenate([shared[rng.integers(0, 500, s)] for s in sizes])  # equal keys within and across maps
    vals = np.arange(keys.size, dtype=np.int64)
    seeds = W.key_stream(56, sizes.size)
    S = F.fks_build_batched(F.FKS_KEY_U64, dev(keys), None, None, seg, seeds, dev(vals), F.make_opts(dedup=1))
    assert (S.status == 0).all()
    keep = O.dedup_keep(keys=keys, seg=seg).astype(bool)
    for j in range(sizes.size):
        sl = slice(seg[j], seg[j + 1])
        om = O.build_u64(keys[sl][keep[sl]], vals[sl][keep[sl]], seed=int(seeds[j]))
        same_tables(F, S.get(j), om)


def test_malformed_offsets_rejected(F):
    ctx = np.frombuffer(b"abcdefgh", np.uint8)
    offs = np.array([0, 3, 2, 8], np.int64)  # element 1 has a negative length
    with pytest.raises(F.FksError) as e:
        F.fks_build_bytes(dev(ctx), dev(offs), dev(np.arange(3)), 1, F.make_opts(dedup=1))
    assert e.value.status == F.FKS_ERR_INVALID_ARG
