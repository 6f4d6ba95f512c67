"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: published
generator check values, closed forms of the range reduction and of the
polynomial fingerprint, statistical properties the paper's analysis relies
on (universal hashing, Sec. 2.1; expected S = O(n) and at most two expected
level-two trials, Sec. 2.3 analysis), the well-formed and collision-free
properties of a hash-set construction (Sec. 2.2), and brute force against a
Python dict on tiny inputs.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2508_11443_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MASK = (1 << 64) - 1
P61 = (1 << 61) - 1


# ------------------------------------------------------------------ helpers
def np_derive(seed, r, tags, a):
    """Constants for many tags at once, vectorised through numpy (used only to
    check table structure fast; tied to the oracle's own or_derive below)."""
    tags = np.asarray(tags, np.uint64)
    a = np.asarray(a, np.uint64)
    cnt = (np.uint64(r) << np.uint64(48)) | (tags << np.uint64(14)) | (a << np.uint64(2))
    out = []
    for j in range(3):
        with np.errstate(over="ignore"):
            z = np.uint64(seed & MASK) + ((cnt | np.uint64(j)) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        out.append(z)
    return out


def np_hash(c, k):
    k = np.asarray(k, np.uint64)
    with np.errstate(over="ignore"):
        acc = c[0] * (k & np.uint64(0xFFFFFFFF)) + c[1] * (k >> np.uint64(32)) + c[2]
    return acc >> np.uint64(32)


def np_reduce(h, m):
    with np.errstate(over="ignore"):
        return (np.asarray(h, np.uint64) * np.asarray(m, np.uint64)) >> np.uint64(32)


def slot_index(m: O.Map, hkeys):
    """h k of Sec. 2.2 for every key, from the map's descriptors."""
    c1 = [np.uint64(x) for x in O.derive(m.seed, m.round, O.TAG_L1, 0)]
    b = np_reduce(np_hash(c1, hkeys), m.nb).astype(np.int64)
    off, s, att = O.desc_fields(m.desc)
    c2 = np_derive(m.seed, m.round, b.astype(np.uint64), att[b].astype(np.uint64))
    j = off[b] + np_reduce(np_hash(c2, hkeys), (s[b] * s[b]).astype(np.uint64)).astype(np.int64)
    return b, j


def test_numpy_helpers_agree_with_oracle_primitives():
    rng = np.random.default_rng(0)
    for _ in range(50):
        seed, r, tag, a = (int(x) for x in rng.integers(0, 2**63, 4))
        r, tag, a = r % 65536, tag % (1 << 30), a % 4096
        c = O.derive(seed, r, tag, a)
        cn = [int(x[0]) for x in np_derive(seed, r, [tag], [a])]
        assert tuple(cn) == c
        k = int(rng.integers(0, 2**63)) * 2 + 1
        assert O.hash32(c, k) == int(np_hash([np.uint64(x) for x in c], [k])[0])


# ------------------------------------------------------------------ R1: generator
def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_vectors.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 8
    for seed, i, want in rows:
        assert O.splitmix64(int(seed), int(i)) == int(want)


def test_derive_coordinates_are_distinct_streams():
    # different rounds, tags, attempts or constant indices never share a
    # counter, so the constants differ (a dropped field would make them equal)
    seen = set()
    for r in range(3):
        for tag in (0, 1, 7, O.TAG_L1, O.TAG_FP):
            for a in range(3):
                c = O.derive(99, r, tag, a)
                assert len(set(c)) == 3
                for x in c:
                    assert x not in seen
                    seen.add(x)


# ------------------------------------------------------------------ R1: hash family
def test_hash_pair_distribution_is_uniform():
    """Strong universality (Thorup 2015, vector multiply-shift): for fixed
    distinct keys the pair (H(k1), H(k2)) is uniform over random constants.
    Checked on the top 3 bits of each (64 cells) with a chi-square bound; a
    dropped additive constant (H(0) = 0 always) or a dropped word product
    fails this."""
    rng = np.random.default_rng(1)
    pairs = [(0, 1), (5, 5 + (1 << 32)), (0x1234_5678_0000_0000, 0x1234_5679_0000_0000),
             (3, 3 | (1 << 63))]
    for k1, k2 in pairs:
        cells = np.zeros(64, np.int64)
        T = 6400
        seeds = rng.integers(0, 2**63, T)
        for s in seeds:
            c = O.derive(int(s), 0, 5, 0)
            h1, h2 = O.hash32(c, k1), O.hash32(c, k2)
            cells[(h1 >> 29) * 8 + (h2 >> 29)] += 1
        chi2 = ((cells - T / 64) ** 2 / (T / 64)).sum()
        assert chi2 < 120, (k1, k2, chi2)  # 63 dof: p < 1e-5


def test_hash_collision_rate_in_small_range():
    """Universal family: P[reduce(H(k1), m) == reduce(H(k2), m)] ~ 1/m for
    keys that differ only in their low word, only in their high word, or in
    both."""
    rng = np.random.default_rng(2)
    m = 16
    for k1, k2 in [(10, 11), (10, 10 + (7 << 32)), (2**63 + 1, 2**62 + 9)]:
        T = 4000
        coll = 0
        for s in rng.integers(0, 2**63, T):
            c = O.derive(int(s), 1, 3, 2)
            coll += O.reduce(O.hash32(c, k1), m) == O.reduce(O.hash32(c, k2), m)
        assert abs(coll / T - 1 / m) < 0.03, (k1, k2, coll / T)


# ------------------------------------------------------------------ R2: reduction
def test_reduce_closed_forms():
    rng = np.random.default_rng(3)
    hs = [0, 1, 2**31, 2**32 - 1] + [int(x) for x in rng.integers(0, 2**32, 200)]
    for h in hs:
        for j in range(0, 33):
            assert O.reduce(h, 1 << j) == h >> (32 - j)     # power-of-two ranges
        for m in (1, 3, 10, 1000, 2**32 - 5, 2**32):
            r = O.reduce(h, m)
            assert 0 <= r < m
            assert r == (h * m) // 2**32                      # floor(h m / 2^32)
    # the preimage of each target t is [ceil(t 2^32 / m), ceil((t+1) 2^32 / m))
    for m in (3, 7, 1000):
        for t in (0, 1, m - 1):
            lo = -(-t * 2**32 // m)
            assert O.reduce(lo, m) == t
            if lo > 0:
                assert O.reduce(lo - 1, m) == t - 1


# ------------------------------------------------------------------ R8: fingerprint
def poly_closed_form(data: bytes, base: int) -> int:
    words = [len(data)] + [int.from_bytes(data[t:t + 4].ljust(4, b"\0"), "little")
                           for t in range(0, len(data), 4)]
    m = len(words)
    return sum(w * pow(base, m - 1 - i, P61) for i, w in enumerate(words)) % P61


def test_fingerprint_matches_closed_form():
    rng = np.random.default_rng(4)
    bases = [1, 2, P61 - 1, O.fp_base(7, 0), O.fp_base(7, 1)]
    for base in bases:
        for L in [0, 1, 3, 4, 5, 8, 17, 64, 200]:
            data = bytes(rng.integers(0, 256, L, dtype=np.uint8))
            assert O.fingerprint(data, base) == poly_closed_form(data, base)
    assert O.fingerprint(b"", 12345) == 0
    # worst-case operands of the 61-bit product
    big = bytes([0xFF] * 40)
    assert O.fingerprint(big, P61 - 1) == poly_closed_form(big, P61 - 1)


def test_fingerprint_base_range_and_round_dependence():
    bases = {O.fp_base(s, r) for s in range(20) for r in range(4)}
    assert all(1 <= b <= P61 - 1 for b in bases)
    assert len(bases) == 80


def test_fingerprint_separates_padding_and_length():
    base = O.fp_base(1, 0)
    assert O.fingerprint(b"ab", base) != O.fingerprint(b"ab\0", base)
    assert O.fingerprint(b"abcd", base) != O.fingerprint(b"abcd\0\0\0\0", base)


# ------------------------------------------------------------------ construction
def check_table(m: O.Map, keys, vals, bound=None):
    """Well-formed and collision-free (Sec. 2.2), S bound, layout, fill rule."""
    n = len(keys)
    lam = m.keys_per_bucket
    bound = bound or 2 * (1 + lam)
    off, s, att = O.desc_fields(m.desc)
    assert m.status == O.OK
    assert m.nb == -(-n // lam) == s.size
    assert s.sum() == n
    assert m.S == int((s * s).sum()) <= bound * n
    # offsets = exclusive presum of shape^2
    assert off[0] == 0 and np.array_equal(off[1:], np.cumsum(s * s)[:-1])
    assert (att[s <= 1] == 0).all()
    b, j = slot_index(m, keys)
    # the level-one histogram is Hist nb (Map g K)
    assert np.array_equal(np.bincount(b, minlength=m.nb), s)
    assert (j >= 0).all() and (j < m.S).all()            # property 1
    assert np.unique(j).size == n                         # property 2
    assert np.array_equal(m.slots[j, 0], np.asarray(keys, np.uint64))
    if m.slots.shape[1] == 2:
        assert np.array_equal(m.slots[j, 1].astype(np.int64), np.asarray(vals, np.int64))
    used = np.zeros(m.S, bool)
    used[j] = True
    # R7: empty slots carry the lowest occupied slot of their bucket, value -1
    for bb in np.nonzero(s >= 2)[0][:2000]:
        lo, hi = off[bb], off[bb] + s[bb] ** 2
        occ = np.nonzero(used[lo:hi])[0]
        first = lo + occ[0]
        for jj in range(lo, hi):
            if not used[jj]:
                assert m.slots[jj, 0] == m.slots[first, 0]
                assert m.slots[jj, -2 if m.slots.shape[1] == 4 else 1] == np.uint64(MASK)
    return b, j


@pytest.mark.parametrize("n", [1, 2, 3, 16, 1000, 1 << 16])
def test_build_invariants(n):
    w = W.u64_workload(n, 2 * n, 0.5, seed=n + 11)
    m = O.build_u64(w.keys, w.vals, seed=77)
    check_table(m, w.keys, w.vals)
    out, found = O.lookup_u64(m, w.queries, absent=-7)
    assert np.array_equal(found, w.expect_found)
    assert np.array_equal(out, np.where(w.expect_found == 1, w.expect_vals, -7))


STRUCTURED = list(W.STRUCTURED_KINDS)


@pytest.mark.parametrize("kind", STRUCTURED)
def test_structured_key_sets(kind):
    keys = W.structured_keys(kind, 4096)
    vals = np.arange(keys.size, dtype=np.int64) * 3 - 5
    m = O.build_u64(keys, vals, seed=19)
    assert m.status == O.OK and m.S <= 4 * keys.size
    check_table(m, keys, vals)
    others = np.setdiff1d(W.structured_keys(kind, 8192), keys)[:1000]
    out, found = O.lookup_u64(m, np.concatenate([keys, others]), absent=-9)
    assert found[: keys.size].all() and not found[keys.size:].any()
    assert np.array_equal(out[: keys.size], vals) and (out[keys.size:] == -9).all()


def test_n1_special_case():
    m = O.build_u64([123456789], [5], seed=1)
    assert m.S == 1 and m.desc[0] == np.uint64(1 << 32)
    assert m.slots[0, 0] == 123456789 and m.slots[0, 1] == 5


def test_first_successful_attempt_is_kept():
    keys = W.key_stream(5, 3000)
    m = O.build_u64(keys, np.arange(3000), seed=3)
    off, s, att = O.desc_fields(m.desc)
    b, _ = slot_index(m, keys)
    checked = 0
    for bb in np.nonzero(att > 0)[0][:200]:
        members = keys[b == bb]
        for a in range(att[bb]):
            c = [np.uint64(x) for x in O.derive(m.seed, m.round, int(bb), a)]
            jj = np_reduce(np_hash(c, members), np.uint64(s[bb] ** 2))
            assert np.unique(jj).size < members.size  # every earlier attempt collides
        checked += 1
    assert checked > 10


def test_brute_force_against_dict():
    rng = np.random.default_rng(5)
    for trial in range(300):
        n = int(rng.integers(1, 65))
        keys = np.unique(rng.integers(0, 2**64, n, dtype=np.uint64, endpoint=False))
        rng.shuffle(keys)
        vals = rng.integers(-2**62, 2**62, keys.size)
        m = O.build_u64(keys, vals, seed=int(rng.integers(0, 2**63)))
        d = dict(zip(keys.tolist(), vals.tolist()))
        probes = np.concatenate([keys, rng.integers(0, 2**64, 64, dtype=np.uint64)])
        out, found = O.lookup_u64(m, probes, absent=-1)
        for q, v, f in zip(probes.tolist(), out.tolist(), found.tolist()):
            assert f == (q in d)
            assert v == d.get(q, -1)


def test_statistics_match_the_analysis():
    """Sec. 2.3: E[sum s^2] = O(n) (2n - 1 for n random buckets) and at most 2
    expected trials per bucket (mean attempt index <= 1)."""
    n = 4096
    ratios, att_means = [], []
    for seed in range(40):
        keys = W.key_stream(1000 + seed, n)
        m = O.build_u64(keys, np.arange(n), seed=seed)
        if m.rounds_used == 1:
            ratios.append(m.S / n)
        off, s, att = O.desc_fields(m.desc)
        att_means.append(att[s >= 2].mean())
    assert abs(np.mean(ratios) - (2 - 1 / n)) < 0.03
    assert np.mean(att_means) < 1.0


def test_duplicates_are_rejected():
    keys = W.key_stream(9, 500)
    dup = keys.copy()
    dup[123] = dup[45]
    assert O.build_u64(dup, np.arange(500), seed=1).status == O.DUPLICATE_KEY
    # every key equal: the space bound fails every round, the global test decides
    assert O.build_u64(np.full(100, 42, np.uint64), np.arange(100), seed=1).status == O.DUPLICATE_KEY
    assert O.build_u64(np.full(2, 42, np.uint64), np.arange(2), seed=1).status == O.DUPLICATE_KEY


def test_forced_reseed_and_failure():
    # bound 1 admits S = n only (all buckets singletons): rounds are redrawn
    keys = W.key_stream(4, 3)
    m = O.build_u64(keys, np.arange(3), seed=2, bound_factor=1, round_cap=200)
    assert m.status == O.OK and m.S == 3 and m.rounds_used >= 1
    many = [O.build_u64(keys, np.arange(3), seed=s, bound_factor=1, round_cap=200).rounds_used
            for s in range(30)]
    assert max(many) > 1
    # no duplicates and an unreachable bound: BUILD_FAILED after round_cap
    m = O.build_u64(W.key_stream(4, 400), np.arange(400), seed=2, bound_factor=1, round_cap=3)
    assert m.status == O.BUILD_FAILED and m.rounds_used == 3


def test_forced_level_two_retries():
    keys = W.key_stream(6, 2000)
    m0 = O.build_u64(keys, np.arange(2000), seed=8)
    m = O.build_u64(keys, np.arange(2000), seed=8, reject_attempts=5)
    off, s, att = O.desc_fields(m.desc)
    assert (att[s >= 2] >= 5).all() and (att[s <= 1] == 0).all()
    check_table(m, keys, np.arange(2000))
    # past the duplicate check point with no duplicates present
    m = O.build_u64(keys, np.arange(2000), seed=8, reject_attempts=70)
    off, s, att = O.desc_fields(m.desc)
    assert m.status == O.OK and (att[s >= 2] >= 70).all()
    assert m0.round == m.round


def test_attempt_cap_moves_to_next_round():
    keys = W.key_stream(6, 300)
    m = O.build_u64(keys, np.arange(300), seed=8, reject_attempts=10, attempt_cap=10, round_cap=4)
    assert m.status == O.BUILD_FAILED  # every round exhausts its attempts


# ------------------------------------------------------------------ strings
def test_string_build_and_lookup():
    w = W.string_workload(3000, 6000, 0.5, seed=3)
    m = O.build_bytes(w.ctx, w.offs, w.vals, seed=12)
    assert m.status == O.OK
    fps = O.fingerprints(w.ctx, w.offs, 12, m.round)
    b, j = check_table(m, fps, w.vals)
    # slot payload: offset and length of the member in the map's context
    lens = np.diff(w.offs)
    assert np.array_equal(m.slots[j, 1], (w.offs[:-1] | (lens << 40)).astype(np.uint64))
    assert np.array_equal(m.slots[j, 2].astype(np.int64), w.vals)
    assert (m.slots[:, 3] == 0).all()
    # needles from a different context (Sec. 3.1)
    out, found = O.lookup_bytes(m, w.qctx, w.qoffs, absent=-3)
    assert np.array_equal(found, w.expect_found)
    assert np.array_equal(out, np.where(w.expect_found == 1, w.expect_vals, -3))


def test_string_fingerprints_are_closed_form():
    w = W.string_workload(200, 10, 0.5, seed=4)
    fps = O.fingerprints(w.ctx, w.offs, 5, 2)
    base = O.fp_base(5, 2)
    for i in range(200):
        assert int(fps[i]) == poly_closed_form(bytes(w.ctx[w.offs[i]:w.offs[i + 1]]), base)


def test_string_duplicates_and_empty_strings():
    ctx = np.frombuffer(b"abcabcxyz", np.uint8)
    offs = np.array([0, 3, 6, 9])
    assert O.build_bytes(ctx, offs, np.arange(3), seed=1).status == O.DUPLICATE_KEY
    # one empty string is a valid key; two are duplicates
    offs2 = np.array([0, 0, 3, 9])
    m = O.build_bytes(ctx, offs2, np.arange(3), seed=1)
    assert m.status == O.OK
    out, found = O.lookup_bytes(m, np.frombuffer(b"abcq", np.uint8), np.array([0, 0, 3, 4]))
    assert found.tolist() == [1, 1, 0] and out.tolist() == [0, 1, -1]
    assert O.build_bytes(ctx, np.array([0, 0, 0, 9]), np.arange(3), seed=1).status == O.DUPLICATE_KEY


def test_string_brute_force():
    rng = np.random.default_rng(6)
    for trial in range(100):
        n = int(rng.integers(1, 40))
        strs = list({bytes(rng.integers(97, 100, int(rng.integers(0, 6)), dtype=np.uint8))
                     for _ in range(n)})
        offs = np.zeros(len(strs) + 1, np.int64)
        offs[1:] = np.cumsum([len(s) for s in strs])
        ctx = np.frombuffer(b"".join(strs) + b"\0", np.uint8)
        vals = rng.integers(-1000, 1000, len(strs))
        m = O.build_bytes(ctx, offs, vals, seed=trial)
        assert m.status == O.OK
        d = dict(zip(strs, vals.tolist()))
        probes = strs + [bytes(rng.integers(97, 100, int(rng.integers(0, 6)), dtype=np.uint8))
                         for _ in range(20)]
        qo = np.zeros(len(probes) + 1, np.int64)
        qo[1:] = np.cumsum([len(s) for s in probes])
        out, found = O.lookup_bytes(m, np.frombuffer(b"".join(probes) + b"\0", np.uint8), qo)
        for p, v, f in zip(probes, out.tolist(), found.tolist()):
            assert f == (p in d) and v == d.get(p, -1)


def test_binary_search_matches_searchsorted():
    rng = np.random.default_rng(7)
    a = np.sort(np.unique(rng.integers(0, 2**64, 1000, dtype=np.uint64)))
    for q in np.concatenate([a[::7], rng.integers(0, 2**64, 100, dtype=np.uint64)]):
        i = int(np.searchsorted(a, q))
        want = i if i < a.size and a[i] == q else -1
        assert O.binary_search(a, int(q)) == want


# ------------------------------------------------------------------ bucket-count variant
# nb = ceil(n / lambda) level-one buckets instead of n; everything else is
# the paper's construction.  The FKS analysis gives E[sum s^2] = n + n (n - 1)
# / nb for a random level-one hash, and the default bound 2 (1 + lambda) n.
@pytest.mark.parametrize("lam", [2, 4, 8, 16])
@pytest.mark.parametrize("n", [1, 5, 17, 1000, 4099, 1 << 15])
def test_bucket_variant_invariants(lam, n):
    w = W.u64_workload(n, 2 * n, 0.5, seed=n + lam)
    m = O.build_u64(w.keys, w.vals, seed=lam * 7 + 1, keys_per_bucket=lam)
    assert m.nb == (n + lam - 1) // lam and m.desc.size == m.nb
    check_table(m, w.keys, w.vals)
    out, found = O.lookup_u64(m, w.queries, absent=-7)
    assert np.array_equal(found, w.expect_found)
    assert np.array_equal(out, np.where(w.expect_found == 1, w.expect_vals, -7))


def test_bucket_variant_lambda1_is_the_paper_build():
    w = W.u64_workload(3000, 10, 0.5, seed=3)
    a = O.build_u64(w.keys, w.vals, seed=9)
    b = O.build_u64(w.keys, w.vals, seed=9, keys_per_bucket=1, bound_factor=4)
    assert a.nb == b.nb == 3000
    assert np.array_equal(a.desc, b.desc) and np.array_equal(a.slots, b.slots)


@pytest.mark.parametrize("lam", [2, 4, 8, 16])
def test_bucket_variant_statistics(lam):
    """Mean S / n over seeds against 1 + (n - 1) / nb; a reduction over n
    buckets instead of nb would give about 2."""
    n = 4096
    nb = n // lam
    ratios = []
    for seed in range(30):
        keys = W.key_stream(500 + seed, n)
        m = O.build_u64(keys, np.arange(n), seed=seed, keys_per_bucket=lam)
        assert m.status == O.OK
        if m.rounds_used == 1:
            ratios.append(m.S / n)
    expect = 1 + (n - 1) / nb
    assert abs(np.mean(ratios) - expect) < 0.04 * expect


@pytest.mark.parametrize("lam", [2, 8, 16])
def test_bucket_variant_brute_force(lam):
    rng = np.random.default_rng(lam)
    for trial in range(120):
        n = int(rng.integers(1, 97))
        keys = np.unique(rng.integers(0, 2**64, n, dtype=np.uint64, endpoint=False))
        rng.shuffle(keys)
        vals = rng.integers(-2**62, 2**62, keys.size)
        m = O.build_u64(keys, vals, seed=int(rng.integers(0, 2**63)), keys_per_bucket=lam)
        assert m.status == O.OK
        d = dict(zip(keys.tolist(), vals.tolist()))
        probes = np.concatenate([keys, rng.integers(0, 2**64, 64, dtype=np.uint64)])
        out, found = O.lookup_u64(m, probes, absent=-1)
        for q, v, f in zip(probes.tolist(), out.tolist(), found.tolist()):
            assert f == (q in d)
            assert v == d.get(q, -1)


def test_bucket_variant_l1_counts_and_bounds():
    keys = W.key_stream(8, 5000)
    for lam in (1, 4, 16):
        nb = -(-5000 // lam)
        cnt = O.l1_counts(keys, seed=4, round_=2, nb=nb)
        c1 = [np.uint64(x) for x in O.derive(4, 2, O.TAG_L1, 0)]
        b = np_reduce(np_hash(c1, keys), np.uint64(nb)).astype(np.int64)
        assert np.array_equal(cnt, np.bincount(b, minlength=nb))
    # a bound below E[S] / n forces redraws; far below it, failure
    m = O.build_u64(keys[:300], np.arange(300), seed=1, keys_per_bucket=8, bound_factor=9, round_cap=200)
    assert m.status == O.OK and m.S <= 9 * 300 and m.rounds_used >= 1
    m = O.build_u64(keys[:300], np.arange(300), seed=1, keys_per_bucket=8, bound_factor=2, round_cap=5)
    assert m.status == O.BUILD_FAILED
    # sizes outside what the descriptor encodes
    assert O.build_u64(keys[:10], np.arange(10), seed=1, keys_per_bucket=17).status == O.INVALID_ARG
    assert O.build_u64(keys[:10], np.arange(10), seed=1, keys_per_bucket=3).status == O.OK


@pytest.mark.parametrize("lam", [4, 16])
def test_bucket_variant_strings(lam):
    w = W.string_workload(3000, 2000, 0.5, seed=lam)
    m = O.build_bytes(w.ctx, w.offs, w.vals, seed=5, keys_per_bucket=lam)
    assert m.status == O.OK and m.nb == -(-3000 // lam)
    out, found = O.lookup_bytes(m, w.qctx, w.qoffs, absent=-3)
    assert np.array_equal(found, w.expect_found)
    assert np.array_equal(out, np.where(w.expect_found == 1, w.expect_vals, -3))


# ------------------------------------------------------------------ from_array (deduplication)
def _first_occurrence_dict(items, segs=None):
    """Independent brute force: a Python set per segment, walked in input order."""
    keep = []
    seen = {}
    for e, k in enumerate(items):
        g = 0 if segs is None else segs[e]
        key = (g, k)
        keep.append(key not in seen)
        seen.setdefault(key, e)
    return np.array(keep, np.uint8)


def test_dedup_u64_first_occurrence():
    rng = np.random.default_rng(11)
    for trial in range(50):
        u = int(rng.integers(1, 400))
        universe = int(rng.integers(1, 50))
        keys = rng.integers(0, universe, u).astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)
        keep = O.dedup_keep(keys=keys)
        assert np.array_equal(keep, _first_occurrence_dict(keys.tolist()))


def test_dedup_strings_and_segments():
    rng = np.random.default_rng(12)
    words = [b"", b"a", b"ab", b"abc", b"b", b"ba", b"abcd" * 5, b"x" * 70]
    for trial in range(30):
        u = int(rng.integers(1, 200))
        pick = [words[i] for i in rng.integers(0, len(words), u)]
        offs = np.concatenate([[0], np.cumsum([len(w) for w in pick])]).astype(np.int64)
        ctx = np.frombuffer(b"".join(pick) + b"\0", np.uint8)[: offs[-1]]
        m = int(rng.integers(1, 5))
        cuts = np.sort(rng.choice(np.arange(1, u), size=min(m - 1, u - 1), replace=False)) if u > 1 else []
        seg = np.concatenate([[0], cuts, [u]]).astype(np.int64)
        segs = np.repeat(np.arange(seg.size - 1), np.diff(seg))
        keep = O.dedup_keep(ctx=ctx, offs=offs, seg=seg)
        assert np.array_equal(keep, _first_occurrence_dict(pick, segs.tolist()))


def test_from_array_lookups_follow_first_occurrence():
    rng = np.random.default_rng(13)
    keys = rng.integers(0, 3000, 10000).astype(np.uint64)
    vals = np.arange(10000, dtype=np.int64)
    m = O.from_array_u64(keys, vals, seed=3)
    assert m.status == O.OK and m.n == np.unique(keys).size
    first = {}
    for e, k in enumerate(keys.tolist()):
        first.setdefault(k, e)
    q = np.arange(3100, dtype=np.uint64)
    out, found = O.lookup_u64(m, q)
    for k, v, f in zip(q.tolist(), out.tolist(), found.tolist()):
        assert f == (k in first) and v == first.get(k, -1)


# ------------------------------------------------------------------ Eytzinger layout
def _inorder(ek, n, k=1, out=None):
    out = [] if out is None else out
    if k <= n:
        _inorder(ek, n, 2 * k, out)
        out.append(int(ek[k]))
        _inorder(ek, n, 2 * k + 1, out)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 15, 100, 1023, 1024, 5000])
def test_eytzinger_layout_is_the_level_order_tree(n):
    rng = np.random.default_rng(n)
    sk = np.sort(np.unique(rng.integers(0, 2**64, n + 50, dtype=np.uint64, endpoint=False)))[:n]
    sv = rng.integers(-2**40, 2**40, n)
    ek, ev = O.eytzinger_layout(sk, sv)
    # a permutation whose in-order walk is the sorted order, values travel with keys
    assert _inorder(ek, n) == sk.tolist()
    pos = {int(k): i for i, k in enumerate(sk.tolist())}
    assert all(ev[k] == sv[pos[int(ek[k])]] for k in range(1, n + 1))
    # heap order: a node is greater than its left child and smaller than its right child
    for k in range(1, n + 1):
        if 2 * k <= n:
            assert ek[2 * k] < ek[k]
        if 2 * k + 1 <= n:
            assert ek[2 * k + 1] > ek[k]


def test_eytzinger_perfect_tree_root_is_the_median():
    for h in range(1, 12):
        n = (1 << h) - 1
        sk = np.arange(n, dtype=np.uint64) * np.uint64(3) + np.uint64(1)
        ek, _ = O.eytzinger_layout(sk, np.arange(n))
        assert ek[1] == sk[n // 2]
        # the last level holds every other key, in order
        assert ek[(n + 1) // 2: n + 1].tolist() == sk[0::2].tolist()


def test_eytzinger_search_matches_binary_search():
    rng = np.random.default_rng(9)
    for n in (1, 2, 3, 10, 777, 4096):
        sk = np.sort(np.unique(rng.integers(0, 1 << 20, n * 2, dtype=np.uint64)))[:n]
        ek, ev = O.eytzinger_layout(sk, np.arange(sk.size))
        for q in rng.integers(0, (1 << 20) + 5, 300, dtype=np.uint64).tolist() + [0, 2**64 - 1] + sk[:5].tolist():
            k = O.eytzinger_search(ek, q)
            i = O.binary_search(sk, q)
            assert (k != 0) == (i >= 0)
            if k:
                assert ek[k] == q and ev[k] == i


# ------------------------------------------------------------------ inline-singleton records
def level_one(m, xs):
    c1 = [np.uint64(x) for x in O.derive(m.seed, m.round, O.TAG_L1, 0)]
    return np_reduce(np_hash(c1, np.asarray(xs, np.uint64)), m.nb).astype(np.int64)


@pytest.mark.parametrize("n", [1, 2, 3, 1000, 20000])
def test_inline_records_follow_their_definition(n):
    """Checked key by key: the bucket of a key that is alone in it holds
    {key, value}; every other bucket holds its own descriptor and a first word
    that hashes to another bucket (so that no needle of the bucket equals it)."""
    w = W.u64_workload(n, 1, 1.0, seed=n + 40)
    m = O.build_u64(w.keys, w.vals, seed=41)
    rec = O.inline_records(m)
    _, s, _ = O.desc_fields(m.desc)
    bk = level_one(m, w.keys)
    one = s[bk] == 1
    assert np.array_equal(rec[bk[one], 0], w.keys[one])
    assert np.array_equal(rec[bk[one], 1].view(np.int64), w.vals[one])
    other = np.nonzero(s != 1)[0]
    assert np.array_equal(rec[other, 1], m.desc[other])
    if m.nb > 1:
        assert (level_one(m, rec[other, 0]) != other).all()
    if n >= 20000:  # P(a key is alone in its bucket) = (1 - 1/n)^(n-1) ~ 1/e
        assert abs(one.mean() - np.exp(-1)) < 0.01


@pytest.mark.parametrize("kind", STRUCTURED + ["random"])
def test_inline_lookup_equals_the_papers_lookup(kind):
    """The record-first lookup answers exactly as the paper's two-probe
    lookup and as a dictionary, members, non-members, 0 and 2^64 - 1."""
    keys = W.key_stream(71, 1500) if kind == "random" else W.structured_keys(kind, 1500)
    vals = np.arange(keys.size, dtype=np.int64) * 7 - 3000
    m = O.build_u64(keys, vals, seed=73)
    rec = O.inline_records(m)
    extra = np.array([0, 2**64 - 1, 1, 2**63], np.uint64)
    q = np.concatenate([keys, W.key_stream(72, 1500), extra])
    oi, fi = O.lookup_u64_inline(m, rec, q, absent=-5)
    op, fp = O.lookup_u64(m, q, absent=-5)
    assert np.array_equal(oi, op) and np.array_equal(fi, fp)
    d = dict(zip(keys.tolist(), vals.tolist()))
    assert [int(f) for f in fi] == [int(x in d) for x in q.tolist()]
    assert oi.tolist() == [d.get(x, -5) for x in q.tolist()]


def test_inline_records_of_a_later_round():
    """A map whose table comes from level-one round >= 1 (a tight space
    bound): the records follow that round's hash."""
    keys = W.key_stream(81, 3000)
    for seed in range(200):
        m = O.build_u64(keys, np.arange(3000), seed=seed, bound_factor=2)
        if m.status == O.OK and m.round >= 1:
            break
    assert m.round >= 1
    rec = O.inline_records(m)
    q = np.concatenate([keys, W.key_stream(82, 500)])
    oi, fi = O.lookup_u64_inline(m, rec, q)
    op, fp = O.lookup_u64(m, q)
    assert np.array_equal(oi, op) and np.array_equal(fi, fp)
