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


# ----------------------------------------------------------------------- serving
U64_MAP_BYTES_PER_KEY = 72     # descriptor 8 B + slot capacity 4 x 16 B
STR_MAP_BYTES_PER_KEY = 136    # descriptor 8 B + slot capacity 4 x 32 B (+ context bytes)


@dataclass
class ServePlan:
    """A request stream: kind 0 = build, 1 = lookup; key_kind 0 = uint64,
    1 = strings.  Builds take map ids 0, 1, ... in order; a map's keys are
    the pool entries [off, off + n).  A lookup of nq needles has nhit members
    of its target map, the rest non-members.  The first `prefill` requests
    are builds."""
    kind: np.ndarray
    key_kind: np.ndarray
    map_id: np.ndarray
    n: np.ndarray
    off: np.ndarray
    seed: np.ndarray
    nq: np.ndarray
    nhit: np.ndarray
    prefill: int
    budget: int


def serving_plan(n_requests: int, seed: int, budget: int, str_offs: np.ndarray, prefill: int = 64,
                 lookup_frac: float = 0.9, hit_frac: float = 0.8, u64_n=(2**10, 2**22),
                 str_n=(2**10, 2**20), nq_range=(1, 2**16), u64_pool: int = 2**22) -> ServePlan:
    """prefill builds, then n_requests requests; lookups target a map drawn
    uniformly from the maps resident at that point, under an LRU model of a
    budget of `budget` bytes (the server's accounted map sizes), so every
    lookup targets a map the server holds."""
    import collections
    rng = np.random.Generator(np.random.PCG64(seed))
    str_pool = str_offs.size - 1
    total = prefill + n_requests
    kind = np.zeros(total, np.uint8)
    key_kind = np.zeros(total, np.uint8)
    map_id = np.zeros(total, np.uint32)
    n = np.zeros(total, np.int64)
    off = np.zeros(total, np.int64)
    sd = np.zeros(total, np.uint64)
    nq = np.zeros(total, np.int64)
    nhit = np.zeros(total, np.int64)
    resident = collections.OrderedDict()   # map id -> bytes, least recent first
    ids, where = [], {}                    # uniform choice among resident maps
    used, next_id = 0, 0

    def drop(mid):
        i = where.pop(mid)
        last = ids.pop()
        if last != mid:
            ids[i] = last
            where[last] = i

    info = {}
    for r in range(total):
        is_build = r < prefill or rng.random() >= lookup_frac or not ids
        if is_build:
            kk = int(rng.random() < 0.5)
            lo, hi = (str_n if kk else u64_n)
            nn = int(np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
            pool = str_pool if kk else u64_pool
            o = int(rng.integers(0, pool - nn + 1))
            need = (STR_MAP_BYTES_PER_KEY * nn + int(str_offs[o + nn] - str_offs[o])) if kk \
                else U64_MAP_BYTES_PER_KEY * nn
            while used + need > budget and resident:
                victim, b = resident.popitem(last=False)
                used -= b
                drop(victim)
            mid = next_id
            next_id += 1
            resident[mid] = need
            used += need
            where[mid] = len(ids)
            ids.append(mid)
            info[mid] = (kk, nn, o)
            kind[r], key_kind[r], map_id[r], n[r], off[r] = 0, kk, mid, nn, o
            sd[r] = np.uint64(rng.integers(0, 2**63))
        else:
            mid = ids[int(rng.integers(0, len(ids)))]
            resident.move_to_end(mid)
            kk, nn, o = info[mid]
            q = int(np.floor(np.exp(rng.uniform(np.log(nq_range[0]), np.log(nq_range[1])))))
            kind[r], key_kind[r], map_id[r], n[r], off[r] = 1, kk, mid, nn, o
            nq[r] = q
            nhit[r] = rng.binomial(q, hit_frac)
    return ServePlan(kind, key_kind, map_id, n, off, sd, nq, nhit, prefill, budget)


def poisson_arrivals_us(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (microseconds from the start) of a Poisson process."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1e6 / rate_per_s, count))


class ServeData:
    """Device payloads of a ServePlan (torch tensors kept alive here) and the
    request descriptors of the C ABI.  Map keys are slices of shared pools:
    uint64 keys of the splitmix stream, strings of a string workload; lookup
    needles are gathered on the device: members drawn uniformly (with
    replacement) from the target map's slice, non-members from pools of
    non-members of every map.  Values of a map are the index of the key in
    the map's slice."""

    def __init__(self, plan: ServePlan, seed: int, u64_pool: int = 2**22, strings=None):
        import torch

        from . import fks as F
        dev = torch.device("cuda")
        self.plan = plan
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        pool = key_stream(seed, u64_pool)
        self.u64_keys = torch.from_numpy(pool.view(np.int64)).to(dev)
        self.u64_vals = torch.arange(u64_pool, dtype=torch.int64, device=dev)
        miss = _non_members(seed, u64_pool, u64_pool)
        self.u64_miss = torch.from_numpy(miss.view(np.int64)).to(dev)
        s = strings
        self.s_ctx = torch.from_numpy(s.ctx).to(dev)
        self.s_offs_h = s.offs
        self.s_offs = torch.from_numpy(s.offs).to(dev)
        self.s_vals = torch.arange(s.offs.size - 1, dtype=torch.int64, device=dev)
        self.m_ctx = torch.from_numpy(s.qctx).to(dev)     # non-member strings
        self.m_offs = torch.from_numpy(s.qoffs).to(dev)
        P = plan
        builds = np.nonzero(P.kind == 0)[0]
        looks = np.nonzero(P.kind == 1)[0]
        # per-build relative offsets of string maps, one tensor
        sb = builds[P.key_kind[builds] == 1]
        rel_len = (P.n[sb] + 1).astype(np.int64)
        rel_start = np.concatenate([[0], np.cumsum(rel_len)[:-1]]) if sb.size else np.zeros(0, np.int64)
        self.rel_offs = torch.empty(int(rel_len.sum()), dtype=torch.int64, device=dev)
        for k, r in enumerate(sb):
            o, nn = int(P.off[r]), int(P.n[r])
            self.rel_offs[rel_start[k]:rel_start[k] + nn + 1] = self.s_offs[o:o + nn + 1] - self.s_offs[o]
        # uint64 needles of all uint64 lookups, gathered at once
        ul = looks[P.key_kind[looks] == 0]
        self.u_q, self.u_start, self.u_hit = self._gather_u64(P, ul, g, dev)
        # string needles of all string lookups: one CSR over every request
        sl = looks[P.key_kind[looks] == 1]
        self.s_qctx, self.s_qoffs, self.s_start, self.s_hit, self.s_idx = self._gather_str(P, sl, g, dev)
        nq_total = int(P.nq[looks].sum()) if looks.size else 0
        self.out = torch.empty(max(nq_total, 1), dtype=torch.int64, device=dev)
        self.found = torch.empty(max(nq_total, 1), dtype=torch.uint8, device=dev)
        out_start = np.zeros(P.kind.size, np.int64)
        if looks.size:
            out_start[looks] = np.concatenate([[0], np.cumsum(P.nq[looks])[:-1]])
        self.out_start = out_start
        # request descriptors
        reqs = (F.fks_request * P.kind.size)()
        ub = {int(r): k for k, r in enumerate(sb)}
        u_index = {int(r): k for k, r in enumerate(ul)}
        s_index = {int(r): k for k, r in enumerate(sl)}
        for r in range(P.kind.size):
            q = reqs[r]
            q.struct_size = ctypes_sizeof_request()
            q.map_id = int(P.map_id[r])
            q.key_kind = int(P.key_kind[r])
            o, nn = int(P.off[r]), int(P.n[r])
            if P.kind[r] == 0:
                q.type = F.FKS_REQ_BUILD
                q.n = nn
                q.seed = int(P.seed[r])
                if P.key_kind[r] == 0:
                    q.val_type = F.FKS_VAL_I64
                    q.keys = self.u64_keys.data_ptr() + 8 * o
                    q.vals = self.u64_vals.data_ptr()
                else:
                    q.val_type = F.FKS_VAL_I64
                    base = int(self.s_offs_h[o])
                    q.ctx = self.s_ctx.data_ptr() + base
                    q.ctx_bytes = int(self.s_offs_h[o + nn]) - base
                    q.offs = self.rel_offs.data_ptr() + 8 * int(rel_start[ub[r]])
                    q.vals = self.s_vals.data_ptr()
            else:
                q.type = F.FKS_REQ_LOOKUP
                q.nq = int(P.nq[r])
                q.absent = -1
                q.out_vals = self.out.data_ptr() + 8 * int(out_start[r])
                q.out_found = self.found.data_ptr() + int(out_start[r])
                if P.key_kind[r] == 0:
                    q.q = self.u_q.data_ptr() + 8 * int(self.u_start[u_index[r]])
                else:
                    q.qctx = self.s_qctx.data_ptr()
                    q.qoffs = self.s_qoffs.data_ptr() + 8 * int(self.s_start[s_index[r]])
        self.reqs = reqs
        self.u_index, self.s_index = u_index, s_index

    def _gather_u64(self, P, rows, g, dev):
        import torch
        if rows.size == 0:
            z = torch.zeros(1, dtype=torch.int64, device=dev)
            return z, np.zeros(0, np.int64), torch.zeros(1, dtype=torch.bool, device=dev)
        nq = torch.from_numpy(P.nq[rows]).to(dev)
        req = torch.repeat_interleave(torch.arange(rows.size, device=dev), nq)
        start = torch.cumsum(nq, 0) - nq
        pos = torch.arange(req.numel(), device=dev) - start[req]
        hit = pos < torch.from_numpy(P.nhit[rows]).to(dev)[req]
        rnd = torch.randint(0, 2**62, (req.numel(),), device=dev, generator=g)
        n = torch.from_numpy(P.n[rows]).to(dev)[req]
        off = torch.from_numpy(P.off[rows]).to(dev)[req]
        hidx = off + rnd % n
        midx = rnd % self.u64_miss.numel()
        q = torch.where(hit, self.u64_keys[hidx], self.u64_miss[midx])
        self.u_expect = torch.where(hit, hidx - off, torch.full_like(hidx, -1))
        return q, start.cpu().numpy(), hit

    def _gather_str(self, P, rows, g, dev):
        import torch
        if rows.size == 0:
            z = torch.zeros(2, dtype=torch.int64, device=dev)
            return torch.zeros(1, dtype=torch.uint8, device=dev), z, np.zeros(0, np.int64), \
                torch.zeros(1, dtype=torch.bool, device=dev), z
        nq = torch.from_numpy(P.nq[rows]).to(dev)
        req = torch.repeat_interleave(torch.arange(rows.size, device=dev), nq)
        start = torch.cumsum(nq, 0) - nq
        pos = torch.arange(req.numel(), device=dev) - start[req]
        hit = pos < torch.from_numpy(P.nhit[rows]).to(dev)[req]
        rnd = torch.randint(0, 2**62, (req.numel(),), device=dev, generator=g)
        n = torch.from_numpy(P.n[rows]).to(dev)[req]
        off = torch.from_numpy(P.off[rows]).to(dev)[req]
        hidx = off + rnd % n
        midx = rnd % (self.m_offs.numel() - 1)
        idx = torch.where(hit, hidx, midx)
        src_start = torch.where(hit, self.s_offs[idx], self.m_offs[idx])
        lens = torch.where(hit, self.s_offs[idx + 1] - self.s_offs[idx], self.m_offs[idx + 1] - self.m_offs[idx])
        qoffs = torch.zeros(idx.numel() + 1, dtype=torch.int64, device=dev)
        qoffs[1:] = torch.cumsum(lens, 0)
        qctx = torch.empty(int(qoffs[-1]), dtype=torch.uint8, device=dev)
        self.s_expect = torch.where(hit, hidx - off, torch.full_like(hidx, -1))
        # gather the bytes in chunks of strings (bounded index tensors)
        chunk = 1 << 22
        for a in range(0, idx.numel(), chunk):
            b = min(idx.numel(), a + chunk)
            ln = lens[a:b]
            dst0 = qoffs[a:b]
            which = torch.repeat_interleave(torch.arange(b - a, device=dev), ln)
            within = torch.arange(which.numel(), device=dev) - (dst0 - qoffs[a])[which]
            srcpos = src_start[a:b][which] + within
            h = hit[a:b][which]
            bytes_ = torch.where(h, self.s_ctx[srcpos.clamp(max=self.s_ctx.numel() - 1)],
                                 self.m_ctx[srcpos.clamp(max=self.m_ctx.numel() - 1)])
            qctx[int(qoffs[a]):int(qoffs[b])] = bytes_
        # per-request CSR slices share one offsets array: a request starting at
        # string s uses qoffs[s .. s + nq] (absolute offsets into qctx)
        return qctx, qoffs, start.cpu().numpy(), hit, idx


def ctypes_sizeof_request() -> int:
    import ctypes

    from . import fks as F
    return ctypes.sizeof(F.fks_request)


STRUCTURED_KINDS = ("consecutive", "high_half", "both_halves", "bits", "top")


def structured_keys(kind: str, n: int) -> np.ndarray:
    """Distinct uint64 key sets with structure that a hash of the two 32-bit
    halves must still spread: consecutive integers 0..n-1; i << 32 (equal low
    halves); i * (2^32 + 1) (equal halves); the 64 single-bit keys, their
    complements and zero (n ignored); 2^64 - 1 - i (the top of the range)."""
    i = np.arange(n, dtype=np.uint64)
    if kind == "consecutive":
        return i
    if kind == "high_half":
        return i << np.uint64(32)
    if kind == "both_halves":
        return i * np.uint64(2**32 + 1)
    if kind == "bits":
        b = np.uint64(1) << np.arange(64, dtype=np.uint64)
        return np.concatenate([b, ~b, np.zeros(1, np.uint64)])
    if kind == "top":
        return np.uint64(2**64 - 1) - i
    raise ValueError(f"unknown key set {kind}")
