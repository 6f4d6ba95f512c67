"""Seeded synthetic inputs shaped like the paper's benchmark workloads.

The paper measures on uniformly distributed distinct 64-bit integer keys and
on distinct 5-25 character strings, with 32-bit values (Sec. 4); the
workloads here keep that shape at the sizes of the benchmark configurations:

* ``u64_workload``     distinct uint64 keys, int64 values = insertion index,
                       a shuffled query mix of members and exact non-members;
* ``string_workload``  distinct lowercase strings of uniform length in
                       [lo, hi] as one byte buffer plus int64 offsets (CSR),
                       with a member / non-member query mix;
* ``batched_workload`` many independent maps of log-uniform sizes given as
                       segment offsets, with (map_id, key) queries.

This module is the input recipe only.  It holds none of the method's
arithmetic (no hashing, no table layout); the device library and the oracle
both receive its arrays as plain inputs.

Key stream: the splitmix64 generator, x_i = mix(seed + (i + 1) * gamma).
``mix`` is a bijection of 64-bit words and gamma is odd, so the first 2^64
outputs are pairwise distinct: no duplicate rejection ever fires for the
integer workloads.  Non-members are drawn from a second stream and tested for
membership exactly by inverting ``mix``.  Index sampling and shuffles use
numpy's PCG64 with the same seed.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1
_M1_INV = np.uint64(pow(0xBF58476D1CE4E5B9, -1, 1 << 64))
_M2_INV = np.uint64(pow(0x94D049BB133111EB, -1, 1 << 64))
_GAMMA_INV = np.uint64(pow(0x9E3779B97F4A7C15, -1, 1 << 64))
NONMEMBER_SALT = 0xA5A5A5A5A5A5A5A5


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _unshift(x: np.ndarray, s: int) -> np.ndarray:
    # inverse of y = x ^ (x >> s)
    y = x.copy()
    k = s
    while k < 64:
        y = x ^ (y >> np.uint64(s))
        k += s
    return y


def _unmix(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        x = _unshift(x, 31)
        x = x * _M2_INV
        x = _unshift(x, 27)
        x = x * _M1_INV
        return _unshift(x, 30)


def key_stream(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+n-1 of the splitmix64 stream for `seed`."""
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(seed & _MASK) + i * _GAMMA)


def stream_index(seed, x: np.ndarray) -> np.ndarray:
    """For every x, the 0-based position i with key_stream(seed)[i] == x (as uint64)."""
    with np.errstate(over="ignore"):
        return (_unmix(np.asarray(x, np.uint64)) - np.asarray(seed, np.uint64)) * _GAMMA_INV - np.uint64(1)


def is_member(seed, n, x: np.ndarray) -> np.ndarray:
    """Exact test: is x among the first n outputs of the stream for `seed`?"""
    return stream_index(seed, x) < np.asarray(n, np.uint64)


@dataclass
class U64Workload:
    keys: np.ndarray      # uint64[n], distinct
    vals: np.ndarray      # int64[n] (insertion index)
    queries: np.ndarray   # uint64[nq]
    expect_found: np.ndarray  # uint8[nq]
    expect_vals: np.ndarray   # int64[nq] (index, or -1)
    seed: int


def u64_workload(n: int, nq: int, hit_frac: float, seed: int) -> U64Workload:
    """n distinct keys from the stream, values = index, nq queries of which a
    fraction hit_frac are uniform draws (with replacement) of inserted keys and
    the rest uniform non-members, shuffled."""
    keys = key_stream(seed, n)
    vals = np.arange(n, dtype=np.int64)
    rng = np.random.Generator(np.random.PCG64(seed))
    n_hit = int(round(nq * hit_frac))
    hit_idx = rng.integers(0, n, n_hit, dtype=np.int64) if n > 0 else np.zeros(0, np.int64)
    miss = _non_members(seed, n, nq - n_hit)
    q = np.concatenate([keys[hit_idx], miss])
    ev = np.concatenate([hit_idx, np.full(nq - n_hit, -1, np.int64)])
    perm = rng.permutation(nq)
    q, ev = q[perm], ev[perm]
    return U64Workload(keys, vals, q, (ev >= 0).astype(np.uint8), ev, seed)


def _non_members(seed: int, n: int, count: int) -> np.ndarray:
    out = []
    start, have = 0, 0
    while have < count:
        c = key_stream(seed ^ NONMEMBER_SALT, count - have + 16, start)
        start += c.size
        c = c[~is_member(seed, n, c)]
        out.append(c[: count - have])
        have += out[-1].size
    return np.concatenate(out) if out else np.zeros(0, np.uint64)


@dataclass
class StringWorkload:
    ctx: np.ndarray       # uint8 bytes of all keys
    offs: np.ndarray      # int64[n+1]
    vals: np.ndarray      # int64[n] (insertion index)
    qctx: np.ndarray      # uint8 bytes of all queries
    qoffs: np.ndarray     # int64[nq+1]
    expect_found: np.ndarray
    expect_vals: np.ndarray
    seed: int


def _random_strings(rng, count, lo, hi):
    lens = rng.integers(lo, hi + 1, count, dtype=np.int64)
    offs = np.zeros(count + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    data = rng.integers(ord("a"), ord("z") + 1, int(offs[-1]), dtype=np.uint8)
    return data, offs, lens


def _rows_by_length(data, offs, lens):
    """{L: (indices, void-view rows)} for strings of each length L."""
    out = {}
    for L in np.unique(lens):
        idx = np.nonzero(lens == L)[0]
        pos = offs[idx][:, None] + np.arange(L)[None, :]
        rows = np.ascontiguousarray(data[pos]).view(np.dtype((np.void, int(L)))).ravel()
        out[int(L)] = (idx, rows)
    return out


def string_workload(n: int, nq: int, hit_frac: float, seed: int, lo: int = 4, hi: int = 64
                    ) -> StringWorkload:
    """n distinct strings, length uniform in [lo, hi], bytes uniform over a-z
    (duplicates drawn are rejected, first occurrence kept); nq queries, a
    fraction hit_frac of them uniform members, the rest fresh strings with the
    same length law that are not members."""
    rng = np.random.Generator(np.random.PCG64(seed))
    keep_data, keep_lens = [], []
    seen = {}
    have = 0
    while have < n:
        want = int((n - have) * 1.02) + 64
        data, offs, lens = _random_strings(rng, want, lo, hi)
        groups = _rows_by_length(data, offs, lens)
        keep = np.zeros(want, bool)
        for L, (idx, rows) in groups.items():
            _, first = np.unique(rows, return_index=True)
            first = np.sort(first)
            cand_idx, cand_rows = idx[first], rows[first]
            if L in seen:
                prev = seen[L]
                dup = np.isin(cand_rows, prev)
                cand_idx, cand_rows = cand_idx[~dup], cand_rows[~dup]
                seen[L] = np.concatenate([prev, cand_rows])
            else:
                seen[L] = cand_rows
            keep[cand_idx] = True
        sel = np.nonzero(keep)[0][: n - have]
        starts, ls = offs[sel], lens[sel]
        pos = np.repeat(starts - np.concatenate([[0], np.cumsum(ls)[:-1]]), ls) + np.arange(ls.sum())
        keep_data.append(data[pos])
        keep_lens.append(ls)
        have += sel.size
        if have >= n:
            break
    ctx = np.concatenate(keep_data)
    lens = np.concatenate(keep_lens)[:n]
    offs = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    ctx = ctx[: offs[-1]]
    # rebuild the membership index from exactly the kept keys
    members = {L: rows for L, (idx, rows) in _rows_by_length(ctx, offs, lens).items()}
    member_idx = {L: idx for L, (idx, rows) in _rows_by_length(ctx, offs, lens).items()}
    vals = np.arange(n, dtype=np.int64)

    n_hit = int(round(nq * hit_frac))
    hit_idx = rng.integers(0, n, n_hit, dtype=np.int64)
    # non-members: fresh strings, rejected when they equal a member
    miss_parts, miss_lens, got = [], [], 0
    while got < nq - n_hit:
        want = int((nq - n_hit - got) * 1.02) + 64
        data, o2, l2 = _random_strings(rng, want, lo, hi)
        ok = np.ones(want, bool)
        for L, (idx, rows) in _rows_by_length(data, o2, l2).items():
            if L in members:
                ok[idx] = ~np.isin(rows, members[L])
        sel = np.nonzero(ok)[0][: nq - n_hit - got]
        starts, ls = o2[sel], l2[sel]
        pos = np.repeat(starts - np.concatenate([[0], np.cumsum(ls)[:-1]]), ls) + np.arange(ls.sum())
        miss_parts.append(data[pos])
        miss_lens.append(ls)
        got += sel.size
    miss_data = np.concatenate(miss_parts) if miss_parts else np.zeros(0, np.uint8)
    miss_l = np.concatenate(miss_lens) if miss_lens else np.zeros(0, np.int64)
    # interleave hits and misses in a shuffled order
    q_is_hit = np.concatenate([np.ones(n_hit, bool), np.zeros(nq - n_hit, bool)])
    src = np.concatenate([hit_idx, np.arange(nq - n_hit)])
    perm = rng.permutation(nq)
    q_is_hit, src = q_is_hit[perm], src[perm]
    miss_offs = np.zeros(miss_l.size + 1, np.int64)
    np.cumsum(miss_l, out=miss_offs[1:])
    qlens = np.where(q_is_hit, lens[np.where(q_is_hit, src, 0)], miss_l[np.where(q_is_hit, 0, src)] if miss_l.size else 0)
    qoffs = np.zeros(nq + 1, np.int64)
    np.cumsum(qlens, out=qoffs[1:])
    starts = np.where(q_is_hit, offs[:-1][np.where(q_is_hit, src, 0)],
                      ctx.size + (miss_offs[:-1][np.where(q_is_hit, 0, src)] if miss_l.size else 0))
    pool = np.concatenate([ctx, miss_data])
    pos = np.repeat(starts - qoffs[:-1], qlens) + np.arange(int(qoffs[-1]))
    qctx = pool[pos]
    ev = np.where(q_is_hit, src, -1).astype(np.int64)
    del members, member_idx
    return StringWorkload(ctx, offs, vals, qctx, qoffs, q_is_hit.astype(np.uint8), ev, seed)


@dataclass
class BatchedWorkload:
    keys: np.ndarray      # uint64[total], map j at seg_offs[j]:seg_offs[j+1]
    vals: np.ndarray      # int64[total] (index within its map)
    seg_offs: np.ndarray  # int64[m+1]
    seeds: np.ndarray     # uint64[m] (build seed of each map)
    key_seeds: np.ndarray  # uint64[m] (stream seed of each map's keys)
    q_map: np.ndarray     # uint32[nq]
    q_keys: np.ndarray    # uint64[nq]
    expect_found: np.ndarray
    expect_vals: np.ndarray


def batched_workload(m: int, n_lo: int, n_hi: int, nq: int, hit_frac: float, seed: int
                     ) -> BatchedWorkload:
    """m maps, n_j = floor(exp(U(ln n_lo, ln n_hi))) distinct keys each (map j's
    keys from stream seed + j); nq queries with map_id drawn proportional to
    n_j, a fraction hit_frac hits (uniform keys of that map), the rest
    non-members of that map."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.floor(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), m))).astype(np.int64)
    sizes = np.clip(sizes, n_lo, n_hi)
    seg = np.zeros(m + 1, np.int64)
    np.cumsum(sizes, out=seg[1:])
    key_seeds = (np.uint64(seed) + np.arange(m, dtype=np.uint64)).astype(np.uint64)
    total = int(seg[-1])
    map_of = np.repeat(np.arange(m), sizes)
    local = np.arange(total, dtype=np.int64) - seg[map_of]
    with np.errstate(over="ignore"):
        keys = _mix(key_seeds[map_of] + (local.astype(np.uint64) + np.uint64(1)) * _GAMMA)
    vals = local.astype(np.int64)
    build_seeds = key_stream(seed ^ 0x5EED5EED5EED5EED, m)
    # queries
    q_map = rng.choice(m, size=nq, p=sizes / sizes.sum()).astype(np.uint32)
    hit = rng.random(nq) < hit_frac
    li = (rng.random(nq) * sizes[q_map]).astype(np.int64)
    li = np.minimum(li, sizes[q_map] - 1)
    q = keys[seg[q_map] + li]
    # misses: the non-member stream of each map, rejection-tested exactly
    nm = int((~hit).sum())
    miss_maps = q_map[~hit]
    cand_i = np.arange(nm, dtype=np.uint64)
    with np.errstate(over="ignore"):
        salt_seeds = key_seeds[miss_maps] ^ np.uint64(NONMEMBER_SALT)
        cand = _mix(salt_seeds + (cand_i + np.uint64(1)) * _GAMMA)
    bad = is_member(key_seeds[miss_maps], sizes[miss_maps].astype(np.uint64), cand)
    step = np.uint64(nm + 1)
    while bad.any():
        with np.errstate(over="ignore"):
            cand_i[bad] += step
            cand[bad] = _mix(salt_seeds[bad] + (cand_i[bad] + np.uint64(1)) * _GAMMA)
        bad = is_member(key_seeds[miss_maps], sizes[miss_maps].astype(np.uint64), cand)
    q[~hit] = cand
    ev = np.where(hit, li, -1).astype(np.int64)
    return BatchedWorkload(keys, vals, seg, build_seeds, key_seeds, q_map, q, hit.astype(np.uint8), ev)
