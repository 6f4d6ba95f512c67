"""Parity of byte-string keys held in a context (Sec. 3.1, 3.3) with the oracle:
fingerprints, tables (including the map's context copy) and lookups of
needles that come with a context of their own are bit-exact."""
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
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_build(F, ctx, offs, vals, seed, **opts):
    return F.fks_build_bytes(dev(np.asarray(ctx, np.uint8)), dev(np.asarray(offs, np.int64)), dev(vals),
                             seed, F.make_opts(**opts) if opts else None)


def gpu_lookup(F, m, qctx, qoffs, i64=True, absent=-1):
    import torch
    nq = len(qoffs) - 1
    out = torch.empty(nq, dtype=torch.int64 if i64 else torch.int32, device="cuda")
    found = torch.empty(nq, dtype=torch.uint8, device="cuda")
    F.fks_lookup_bytes(m, dev(np.asarray(qctx, np.uint8)), dev(np.asarray(qoffs, np.int64)), out, found, absent)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int64), found.cpu().numpy()


def assert_same(F, gm, om):
    desc, slots, ctx = F.fks_map_export(gm)
    assert F.fks_map_info(gm).round == om.round
    assert np.array_equal(desc, om.desc)
    assert np.array_equal(slots, om.slots)
    assert np.array_equal(ctx, om.ctx[: ctx.size])


@pytest.mark.parametrize("n", [1, 2, 5, 1000, 3001, 20000])
@pytest.mark.parametrize("i64", [True, False])
def test_string_tables_and_lookups(F, n, i64):
    w = W.string_workload(n, 2 * n + 1, 0.5, seed=n + 3)
    vals = w.vals if i64 else w.vals.astype(np.int32)
    om = O.build_bytes(w.ctx, w.offs, w.vals, seed=n)
    gm = gpu_build(F, w.ctx, w.offs, vals, n)
    assert_same(F, gm, om)
    out, found = gpu_lookup(F, gm, w.qctx, w.qoffs, i64=i64, absent=-9)
    oo, of = O.lookup_bytes(om, w.qctx, w.qoffs, absent=-9)
    assert np.array_equal(found, of) and np.array_equal(out, oo)
    assert np.array_equal(found, w.expect_found)


def test_string_duplicates_empty_and_invalid(F):
    ctx = np.frombuffer(b"abcabcxyz", np.uint8)
    with pytest.raises(F.FksError) as e:
        gpu_build(F, ctx, [0, 3, 6, 9], np.arange(3), 1)
    assert e.value.status == F.FKS_ERR_DUPLICATE_KEY
    om = O.build_bytes(ctx, [0, 0, 3, 9], np.arange(3), seed=1)
    gm = gpu_build(F, ctx, [0, 0, 3, 9], np.arange(3), 1)
    assert_same(F, gm, om)
    out, found = gpu_lookup(F, gm, np.frombuffer(b"abcq", np.uint8), [0, 0, 3, 4])
    assert found.tolist() == [1, 1, 0] and out.tolist() == [0, 1, -1]
    with pytest.raises(F.FksError) as e:
        gpu_build(F, ctx, [0, 0, 0, 9], np.arange(3), 1)
    assert e.value.status == F.FKS_ERR_DUPLICATE_KEY
    with pytest.raises(F.FksError) as e:
        gpu_build(F, ctx, [0, 5, 3, 9], np.arange(3), 1)
    assert e.value.status == F.FKS_ERR_INVALID_ARG
    # many copies of one string: every round fails the space bound
    many = np.frombuffer(b"hello" * 300, np.uint8)
    with pytest.raises(F.FksError) as e:
        gpu_build(F, many, np.arange(0, 1501, 5), np.arange(300), 1)
    assert e.value.status == F.FKS_ERR_DUPLICATE_KEY


def test_unaligned_contexts(F):
    """Keys and needles that start at arbitrary byte offsets of their buffers."""
    import torch
    w = W.string_workload(5000, 7000, 0.5, seed=8)
    om = O.build_bytes(w.ctx, w.offs, w.vals, seed=4)
    ctx_t = dev(np.concatenate([[7, 7, 7], w.ctx]).astype(np.uint8))[3:]
    gm = F.fks_build_bytes(ctx_t, dev(w.offs), dev(w.vals), 4)
    assert_same(F, gm, om)
    q_t = dev(np.concatenate([[1], w.qctx]).astype(np.uint8))[1:]
    out = torch.empty(len(w.qoffs) - 1, dtype=torch.int64, device="cuda")
    found = torch.empty(len(w.qoffs) - 1, dtype=torch.uint8, device="cuda")
    F.fks_lookup_bytes(gm, q_t, dev(w.qoffs), out, found, -1)
    torch.cuda.synchronize()
    oo, of = O.lookup_bytes(om, w.qctx, w.qoffs)
    assert np.array_equal(out.cpu().numpy(), oo) and np.array_equal(found.cpu().numpy(), of)


def test_long_and_binary_strings(F):
    rng = np.random.default_rng(3)
    lens = rng.integers(0, 3000, 300)
    lens[:5] = [0, 1, 2, 3, 65535]
    offs = np.zeros(lens.size + 1, np.int64)
    offs[1:] = np.cumsum(lens)
    ctx = rng.integers(0, 256, int(offs[-1]), dtype=np.uint8)
    om = O.build_bytes(ctx, offs, np.arange(lens.size), seed=5)
    assert om.status == O.OK
    gm = gpu_build(F, ctx, offs, np.arange(lens.size), 5)
    assert_same(F, gm, om)
    out, found = gpu_lookup(F, gm, ctx, offs)
    assert found.all() and np.array_equal(out, np.arange(lens.size))


def test_full_size_2e22_strings(F):
    """2^22 distinct strings (lengths 4..64, a-z), 2^24 needles at 50 % hits."""
    import torch
    w = W.string_workload(1 << 22, 1 << 24, 0.5, seed=3)
    vals = w.vals.astype(np.int32)
    gm = gpu_build(F, w.ctx, w.offs, vals, 3)
    out, found = gpu_lookup(F, gm, w.qctx, w.qoffs, i64=False)
    assert np.array_equal(found, w.expect_found)
    assert np.array_equal(out, np.where(w.expect_found == 1, w.expect_vals, -1))
    om = O.build_bytes(w.ctx, w.offs, w.vals, seed=3)
    assert_same(F, gm, om)
    del gm
    torch.cuda.empty_cache()


def test_short_and_long_strings_in_the_same_warps(F):
    """Strings above 128 bytes are fingerprinted and compared by the whole
    warp, shorter ones by their lane: a mix of both in every warp, members
    and non-members (a long non-member differing from a member only in its
    last byte), against the oracle."""
    rng = np.random.default_rng(11)
    n = 6000
    lens = rng.integers(4, 65, n)
    longs = rng.random(n) < 0.1
    lens[longs] = rng.integers(129, 3000, int(longs.sum()))
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum(lens)
    ctx = rng.integers(0, 256, int(offs[-1]), dtype=np.uint8)
    vals = np.arange(n)
    om = O.build_bytes(ctx, offs, vals, seed=12)
    assert om.status == O.OK
    gm = gpu_build(F, ctx, offs, vals, 12)
    assert_same(F, gm, om)
    # needles: every member, then each long member with its last byte changed
    lk = np.nonzero(longs)[0]
    pieces, qlens = [ctx], list(lens)
    for k in lk:
        s = ctx[offs[k]:offs[k + 1]].copy()
        s[-1] ^= 0x5A
        pieces.append(s)
        qlens.append(s.size)
    qctx = np.concatenate(pieces)
    qoffs = np.zeros(len(qlens) + 1, np.int64)
    qoffs[1:] = np.cumsum(qlens)
    out, found = gpu_lookup(F, gm, qctx, qoffs)
    oo, of = O.lookup_bytes(om, qctx, qoffs)
    assert np.array_equal(found, of) and np.array_equal(out, oo)
    assert found[:n].all() and not found[n:].any()


def test_strings_up_to_the_per_lane_limit(F):
    """Lengths 5..128 bytes (the longest strings a lane still fingerprints and
    compares alone) and one empty string, at an aligned and at an unaligned
    context start: tables (fingerprints included) and lookups equal the
    oracle's."""
    rng = np.random.default_rng(41)
    n = 20000
    lens = rng.integers(5, 129, n)
    lens[777] = 0
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum(lens)
    body = rng.integers(0, 256, int(offs[-1]), dtype=np.uint8)
    vals = np.arange(n)
    om = O.build_bytes(body, offs, vals, seed=14)
    assert om.status == O.OK
    for pad in (0, 3):
        ctx_t = dev(np.concatenate([np.zeros(pad, np.uint8), body]))[pad:]
        gm = F.fks_build_bytes(ctx_t, dev(offs), dev(vals), 14)
        assert_same(F, gm, om)
        out, found = gpu_lookup(F, gm, body, offs)
        assert found.all() and np.array_equal(out, vals)


def test_longest_string_and_size_limits(F):
    """The longest key a map takes (2^24 - 1 bytes) builds with the oracle's
    table and is found; a key one byte longer is refused
    (FKS_ERR_INVALID_ARG), a needle that long is absent without an error, and
    n = 2^30 keys is refused before any device work."""
    import ctypes
    rng = np.random.default_rng(51)
    big = 1 << 24
    lens = np.array([big - 1, 5, 17, 0, 64])
    offs = np.zeros(lens.size + 1, np.int64)
    offs[1:] = np.cumsum(lens)
    ctx = rng.integers(0, 256, int(offs[-1]), dtype=np.uint8)
    vals = np.arange(lens.size)
    om = O.build_bytes(ctx, offs, vals, seed=2)
    assert om.status == O.OK
    gm = gpu_build(F, ctx, offs, vals, 2)
    assert_same(F, gm, om)
    out, found = gpu_lookup(F, gm, ctx, offs)
    assert found.all() and np.array_equal(out, vals)
    needle = np.concatenate([ctx[:big - 1], np.array([7], np.uint8)])  # 2^24 bytes
    out, found = gpu_lookup(F, gm, needle, [0, big])
    assert found.tolist() == [0] and out.tolist() == [-1]
    offs2 = np.array([0, big, big + 5], np.int64)
    ctx2 = rng.integers(0, 256, big + 5, dtype=np.uint8)
    with pytest.raises(F.FksError) as e:
        gpu_build(F, ctx2, offs2, np.arange(2), 2)
    assert e.value.status == F.FKS_ERR_INVALID_ARG
    k = dev(np.zeros(8, np.int64))
    h = ctypes.c_void_p()
    st = F.lib().fks_build_u64(ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(k.data_ptr()), F.FKS_VAL_I64, 1 << 30,
                               1, None, None, None, ctypes.byref(h))
    assert st == F.FKS_ERR_INVALID_ARG and not h.value
