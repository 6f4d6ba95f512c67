"""CPU oracle for the FKS two-level hash map -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
the two share no code: ``fks_oracle.c`` is an independent, plain,
single-threaded C restatement of the paper's functional construction
(``make_1`` / ``make_2``, Sec. 2.3) and of the membership test (Sec. 2.2).

This module compiles that file with gcc (in-tree) and marshals numpy arrays
through ctypes.  It also writes out, in numpy and plain Python, the
inline-singleton records of a built uint64 map and the lookup that reads
them: a transform of the map's own tables, not a second construction.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fks_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

OK, INVALID_ARG, DUPLICATE_KEY, OUT_OF_MEMORY, BUILD_FAILED = 0, 1, 2, 3, 4

_lib = None


def build(force: bool = False) -> str:
    """Compile fks_oracle.c into oracle/liboracle.so (plain -O2, no -ffast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("round", ctypes.c_uint32),
                ("max_s", ctypes.c_uint32), ("S", ctypes.c_uint64), ("c1", ctypes.c_uint64 * 3),
                ("attempts_sum", ctypes.c_uint64), ("nonempty", ctypes.c_uint64),
                ("rounds_used", ctypes.c_uint32), ("max_attempt", ctypes.c_uint32),
                ("nb", ctypes.c_uint64)]


class _Opts(ctypes.Structure):
    _fields_ = [("bound_factor", ctypes.c_uint32), ("round_cap", ctypes.c_uint32),
                ("attempt_cap", ctypes.c_uint32), ("reject_attempts", ctypes.c_uint32),
                ("keys_per_bucket", ctypes.c_uint32)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        L.or_splitmix64.restype = u64
        L.or_splitmix64.argtypes = [u64, u64]
        L.or_derive.restype = None
        L.or_derive.argtypes = [u64, u32, u64, u32, vp]
        L.or_hash.restype = u32
        L.or_hash.argtypes = [vp, u64]
        L.or_reduce.restype = u64
        L.or_reduce.argtypes = [u32, u64]
        L.or_fp_base.restype = u64
        L.or_fp_base.argtypes = [u64, u32]
        L.or_fingerprint.restype = u64
        L.or_fingerprint.argtypes = [vp, u64, u64]
        L.or_build_u64.restype = ctypes.c_int
        L.or_build_u64.argtypes = [vp, vp, u64, u64, vp, vp, vp, u64, vp]
        L.or_build_bytes.restype = ctypes.c_int
        L.or_build_bytes.argtypes = [vp, vp, vp, u64, u64, vp, vp, vp, u64, vp]
        L.or_lookup_u64.restype = None
        L.or_lookup_u64.argtypes = [vp, vp, u64, u64, u32, vp, u64, ctypes.c_int64, vp, vp]
        L.or_lookup_bytes.restype = None
        L.or_lookup_bytes.argtypes = [vp, vp, vp, u64, u64, u32, vp, vp, u64, ctypes.c_int64, vp, vp]
        L.or_l1_counts.restype = None
        L.or_l1_counts.argtypes = [vp, u64, u64, u64, u32, vp]
        L.or_fingerprints.restype = None
        L.or_fingerprints.argtypes = [vp, vp, u64, u64, u32, vp]
        L.or_dedup.restype = u64
        L.or_dedup.argtypes = [vp, vp, vp, u64, vp, u32, vp]
        L.or_eytzinger_layout.restype = None
        L.or_eytzinger_layout.argtypes = [vp, vp, u64, vp, vp]
        L.or_eytzinger_search.restype = u64
        L.or_eytzinger_search.argtypes = [vp, u64, u64]
        L.or_binary_search.restype = ctypes.c_int64
        L.or_binary_search.argtypes = [vp, u64, u64]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


# ------------------------------------------------------------- primitives
def splitmix64(seed: int, i: int) -> int:
    """i-th output of the splitmix64 generator started at `seed`."""
    return int(lib().or_splitmix64(seed & (2**64 - 1), i & (2**64 - 1)))


TAG_L1 = 0xFFFFFFFF
TAG_FP = 0xFFFFFFFE


def derive(seed: int, round_: int, tag: int, attempt: int) -> tuple[int, int, int]:
    out = np.zeros(3, np.uint64)
    lib().or_derive(seed & (2**64 - 1), round_, tag, attempt, _p(out))
    return tuple(int(x) for x in out)


def hash32(c, k: int) -> int:
    cc = _c(c, np.uint64)
    return int(lib().or_hash(_p(cc), k & (2**64 - 1)))


def reduce(h: int, m: int) -> int:
    return int(lib().or_reduce(h, m))


def fp_base(seed: int, round_: int) -> int:
    return int(lib().or_fp_base(seed & (2**64 - 1), round_))


def fingerprint(data: bytes, base: int) -> int:
    buf = np.frombuffer(bytes(data) + b"\0", np.uint8)
    return int(lib().or_fingerprint(_p(buf), len(data), base))


# ------------------------------------------------------------- maps
@dataclass
class Map:
    status: int
    n: int
    seed: int
    round: int = 0
    S: int = 0
    max_s: int = 0
    c1: tuple = ()
    attempts_sum: int = 0
    nonempty: int = 0
    rounds_used: int = 0
    max_attempt: int = 0
    nb: int = 0                         # level-one buckets
    keys_per_bucket: int = 1
    desc: np.ndarray | None = None      # uint64[nb]
    slots: np.ndarray | None = None     # uint64[S, words]
    ctx: np.ndarray | None = None       # strings: the map's own context
    kind: str = "u64"


def buckets(n: int, keys_per_bucket: int = 1) -> int:
    """Level-one buckets of an n-key map: ceil(n / keys_per_bucket)."""
    return -(-n // keys_per_bucket)


def default_bound(keys_per_bucket: int = 1) -> int:
    return 2 * (1 + keys_per_bucket)


def _opts(bound_factor=0, round_cap=32, attempt_cap=4095, reject_attempts=0, keys_per_bucket=1):
    return _Opts(bound_factor or default_bound(keys_per_bucket), round_cap, attempt_cap,
                 reject_attempts, keys_per_bucket)


def _finish(st, info, n, seed, desc, slots, words, kind, ctx=None, lam=1) -> Map:
    m = Map(status=st, n=n, seed=seed, kind=kind, nb=buckets(n, lam) if n else 0,
            keys_per_bucket=lam)
    if st == OK:
        m.round, m.S, m.max_s = int(info.round), int(info.S), int(info.max_s)
        m.c1 = tuple(int(x) for x in info.c1)
        m.attempts_sum, m.nonempty = int(info.attempts_sum), int(info.nonempty)
        m.rounds_used, m.max_attempt = int(info.rounds_used), int(info.max_attempt)
        m.desc = desc
        m.slots = slots[: m.S * words].reshape(m.S, words).copy()
        m.ctx = ctx
    else:
        m.rounds_used = int(info.rounds_used)
    return m


def build_u64(keys, vals, seed: int, **opts) -> Map:
    """Oracle build over uint64 keys with int64 values (int32 values are
    passed sign-extended)."""
    keys = _c(keys, np.uint64)
    vals = _c(vals, np.int64)
    n = keys.size
    o = _opts(**opts)
    lam = max(1, o.keys_per_bucket)
    nb = buckets(n, lam)
    cap = max(1, o.bound_factor * n)
    desc = np.zeros(max(nb, 1), np.uint64)
    slots = np.zeros(2 * cap, np.uint64)
    info = _Info()
    st = lib().or_build_u64(_p(keys), _p(vals), n, seed & (2**64 - 1), ctypes.byref(o), _p(desc),
                            _p(slots), cap, ctypes.byref(info))
    return _finish(st, info, n, seed, desc[:nb], slots, 2, "u64", lam=lam)


def build_bytes(ctx, offs, vals, seed: int, **opts) -> Map:
    """Oracle build over byte-string keys ctx[offs[i]:offs[i+1]]."""
    ctx = _c(ctx, np.uint8)
    if ctx.size == 0:
        ctx = np.zeros(1, np.uint8)
    offs = _c(offs, np.int64)
    vals = _c(vals, np.int64)
    n = offs.size - 1
    o = _opts(**opts)
    lam = max(1, o.keys_per_bucket)
    nb = buckets(n, lam) if n > 0 else 0
    cap = max(1, o.bound_factor * n)
    desc = np.zeros(max(nb, 1), np.uint64)
    slots = np.zeros(4 * cap, np.uint64)
    info = _Info()
    st = lib().or_build_bytes(_p(ctx), _p(offs), _p(vals), n, seed & (2**64 - 1), ctypes.byref(o),
                              _p(desc), _p(slots), cap, ctypes.byref(info))
    return _finish(st, info, n, seed, desc[:nb], slots, 4, "bytes", ctx, lam=lam)


def lookup_u64(m: Map, queries, absent: int = -1):
    q = _c(queries, np.uint64)
    out = np.empty(q.size, np.int64)
    found = np.empty(q.size, np.uint8)
    slots = np.ascontiguousarray(m.slots)
    lib().or_lookup_u64(_p(m.desc), _p(slots), m.nb, m.seed & (2**64 - 1), m.round, _p(q), q.size,
                        absent, _p(out), _p(found))
    return out, found


def lookup_bytes(m: Map, qctx, qoffs, absent: int = -1):
    qctx = _c(qctx, np.uint8)
    if qctx.size == 0:
        qctx = np.zeros(1, np.uint8)
    qoffs = _c(qoffs, np.int64)
    nq = qoffs.size - 1
    out = np.empty(nq, np.int64)
    found = np.empty(nq, np.uint8)
    slots = np.ascontiguousarray(m.slots)
    lib().or_lookup_bytes(_p(m.desc), _p(slots), _p(m.ctx), m.nb, m.seed & (2**64 - 1), m.round,
                          _p(qctx), _p(qoffs), nq, absent, _p(out), _p(found))
    return out, found


def l1_counts(hkeys, seed: int, round_: int, nb: int | None = None) -> np.ndarray:
    """Keys per level-one bucket in round `round_` (nb buckets; default one per key)."""
    k = _c(hkeys, np.uint64)
    nb = k.size if nb is None else nb
    cnt = np.zeros(max(nb, 1), np.uint32)
    lib().or_l1_counts(_p(k), k.size, nb, seed & (2**64 - 1), round_, _p(cnt))
    return cnt[:nb]


def fingerprints(ctx, offs, seed: int, round_: int) -> np.ndarray:
    ctx = _c(ctx, np.uint8)
    if ctx.size == 0:
        ctx = np.zeros(1, np.uint8)
    offs = _c(offs, np.int64)
    out = np.zeros(offs.size - 1, np.uint64)
    lib().or_fingerprints(_p(ctx), _p(offs), offs.size - 1, seed & (2**64 - 1), round_, _p(out))
    return out


def dedup_keep(keys=None, ctx=None, offs=None, seg=None) -> np.ndarray:
    """from_array's first-occurrence rule: keep[e] = 1 iff no earlier element
    of e's segment has an equal key (uint64 keys, or byte strings ctx/offs)."""
    if keys is not None:
        k = _c(keys, np.uint64)
        u = k.size
        kp, cp, op = _p(k), None, None
    else:
        cx = _c(ctx, np.uint8)
        if cx.size == 0:
            cx = np.zeros(1, np.uint8)
        of = _c(offs, np.int64)
        u = of.size - 1
        kp, cp, op = None, _p(cx), _p(of)
    keep = np.zeros(max(u, 1), np.uint8)
    sg = None if seg is None else _c(seg, np.int64)
    lib().or_dedup(kp, cp, op, u, None if sg is None else _p(sg), 0 if sg is None else sg.size - 1,
                   _p(keep))
    return keep[:u]


def from_array_u64(keys, vals, seed: int, **opts) -> Map:
    """from_array over uint64 keys: duplicates allowed, first occurrence wins."""
    keep = dedup_keep(keys=keys).astype(bool)
    return build_u64(np.asarray(keys, np.uint64)[keep], np.asarray(vals, np.int64)[keep], seed, **opts)


def eytzinger_layout(sorted_keys, sorted_vals):
    """(keys, values) in Eytzinger order, 1-based: index 0 is unused (0)."""
    sk = _c(sorted_keys, np.uint64)
    sv = _c(sorted_vals, np.int64)
    n = sk.size
    ek = np.zeros(n + 1, np.uint64)
    ev = np.zeros(n + 1, np.int64)
    lib().or_eytzinger_layout(_p(sk), _p(sv), n, _p(ek), _p(ev))
    return ek, ev


def eytzinger_search(ek, q: int) -> int:
    """Node of q in an Eytzinger array (1-based), or 0 when absent."""
    e = _c(ek, np.uint64)
    return int(lib().or_eytzinger_search(_p(e), e.size - 1, q & (2**64 - 1)))


def binary_search(sorted_keys, q: int) -> int:
    s = _c(sorted_keys, np.uint64)
    return int(lib().or_binary_search(_p(s), s.size, q & (2**64 - 1)))


# ------------------------------------------------------------- table reading
# ------------------------------------------------------------- inline-singleton records
def inline_records(m: Map) -> np.ndarray:
    """The inline-singleton records of a uint64 map (lambda 1), uint64[nb, 2],
    written out from the map's own tables.  Bucket b with one key holds
    {key, value}, the contents of its only slot.  Any other bucket holds
    {x_b, desc[b]}, where x_b is a key of another bucket: 0, except for
    b = g(0), where x_b is the least x >= 1 with g(x) != g(0); g(k) =
    reduce(hash32(c1, k), nb) is the level-one hash of the final round."""
    assert m.kind == "u64" and m.keys_per_bucket == 1 and m.status == OK
    off, s, _ = desc_fields(m.desc)
    g0 = reduce(hash32(m.c1, 0), m.nb)
    x1 = 1
    while m.nb > 1 and x1 < (1 << 16) and reduce(hash32(m.c1, x1), m.nb) == g0:
        x1 += 1
    rec = np.zeros((m.nb, 2), np.uint64)
    rec[g0, 0] = x1
    rec[:, 1] = m.desc
    one = s == 1
    rec[one, 0] = m.slots[off[one], 0]
    rec[one, 1] = m.slots[off[one], 1]
    return rec


def lookup_u64_inline(m: Map, rec: np.ndarray, queries, absent: int = -1):
    """Lookups that read the needle's record first, one needle at a time
    (plain Python, for small inputs).  b = g(q) and {x, y} = rec[b].  If x = q,
    q is the bucket's one key and y its value.  Else, if g(x) = b, the bucket
    holds one other key: q is absent.  Else y is desc[b] and the lookup is the
    paper's (Sec. 2.2): s = 0 means absent; otherwise the slot off + Hash c2 q
    mod s^2 holds q or q is absent."""
    out = np.full(len(queries), absent, np.int64)
    found = np.zeros(len(queries), np.uint8)
    for i, q in enumerate(np.asarray(queries, np.uint64).tolist()):
        b = reduce(hash32(m.c1, q), m.nb)
        x, y = int(rec[b, 0]), int(rec[b, 1])
        if x == q:
            out[i], found[i] = np.uint64(y).view(np.int64), 1
            continue
        if reduce(hash32(m.c1, x), m.nb) == b:
            continue
        off, s, att = y & 0xFFFFFFFF, (y >> 32) & 0xFFFFF, y >> 52
        if s == 0:
            continue
        j = off + reduce(hash32(derive(m.seed, m.round, b, att), q), s * s)
        if int(m.slots[j, 0]) == q:
            out[i], found[i] = m.slots[j, 1].view(np.int64), 1
    return out, found


def desc_fields(desc: np.ndarray):
    """(slot_off, s, attempt) arrays of a descriptor array."""
    d = np.asarray(desc, np.uint64)
    return (d & np.uint64(0xFFFFFFFF)).astype(np.int64), \
        ((d >> np.uint64(32)) & np.uint64(0xFFFFF)).astype(np.int64), \
        (d >> np.uint64(52)).astype(np.int64)
