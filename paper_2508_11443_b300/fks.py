"""Thin Python binding of the C ABI in ``include/fks.h`` (argument marshalling only).

Every function has the name of the C entry point it calls.  Device buffers
are torch CUDA tensors (their ``data_ptr()`` is passed); the stream is the
current torch stream unless one is given.  A non-OK status raises
``FksError`` carrying the status and the library's message.  All work runs
in the compiled library ``libfks.so``; there is no Python or CPU fallback, and
importing this module without the compiled library fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfks.so")

FKS_OK = 0
FKS_ERR_INVALID_ARG = 1
FKS_ERR_DUPLICATE_KEY = 2
FKS_ERR_OUT_OF_MEMORY = 3
FKS_ERR_BUILD_FAILED = 4
FKS_ERR_TIMEOUT = 5
FKS_ERR_CUDA = 6
FKS_ERR_EVICTED = 7
FKS_VAL_I32, FKS_VAL_I64 = 0, 1
FKS_KEY_U64, FKS_KEY_BYTES = 0, 1


class FksError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fks status {status}: {msg}")
        self.status = status


class fks_build_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("bound_factor", ctypes.c_uint32),
                ("attempt_cap", ctypes.c_uint32), ("round_cap", ctypes.c_uint32),
                ("reject_attempts", ctypes.c_uint32), ("spin_limit", ctypes.c_uint32),
                ("keys_per_bucket", ctypes.c_uint32), ("dedup", ctypes.c_uint32),
                ("inline_singletons", ctypes.c_uint32)]


class fks_map_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("slots", ctypes.c_uint64),
                ("slot_capacity", ctypes.c_uint64), ("bytes", ctypes.c_uint64),
                ("attempts_sum", ctypes.c_uint64), ("context_bytes", ctypes.c_uint64),
                ("round", ctypes.c_uint32), ("max_bucket", ctypes.c_uint32),
                ("max_attempt", ctypes.c_uint32), ("key_kind", ctypes.c_uint32),
                ("val_type", ctypes.c_uint32), ("overflow_partitions", ctypes.c_uint32),
                ("nonempty_buckets", ctypes.c_uint64), ("buckets", ctypes.c_uint64),
                ("keys_per_bucket", ctypes.c_uint32), ("inline_singletons", ctypes.c_uint32)]


class fks_build_profile(ctypes.Structure):
    _fields_ = [("fingerprint_ms", ctypes.c_float), ("count_ms", ctypes.c_float),
                ("scan_ms", ctypes.c_float), ("scatter_ms", ctypes.c_float),
                ("part_build_ms", ctypes.c_float), ("passes", ctypes.c_uint32),
                ("grouping_levels", ctypes.c_uint32), ("group_ms", ctypes.c_float)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class fks_allocator(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("user", ctypes.c_void_p)]


class Allocator:
    """A device-memory hook for the library (fks_allocator): alloc(nbytes,
    stream) -> device pointer or 0/None, free(ptr, nbytes, stream).  Keep the
    object alive while any map built with it exists: the library calls free
    when the map is destroyed."""

    def __init__(self, alloc, free):
        self._alloc = ALLOC_FN(lambda n, st, u: alloc(int(n), int(st or 0)) or None)
        self._free = FREE_FN(lambda ptr, n, st, u: free(int(ptr), int(n), int(st or 0)))
        self.struct = fks_allocator(ctypes.sizeof(fks_allocator), self._alloc, self._free, None)

    def ref(self):
        return ctypes.byref(self.struct)


def torch_allocator() -> Allocator:
    """Tables and scratch from torch's caching allocator (stream-ordered on the
    stream the library passes); an allocation failure becomes NULL, which the
    library reports as FKS_ERR_OUT_OF_MEMORY."""
    import torch

    def alloc(n, stream):
        try:
            return torch.cuda.caching_allocator_alloc(n, stream=stream)
        except RuntimeError:
            return None

    def free(ptr, n, stream):
        torch.cuda.caching_allocator_delete(ptr)

    return Allocator(alloc, free)


def _aref(alloc):
    return None if alloc is None else alloc.ref()


_lib = None


def lib():
    """The loaded libfks.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2508_11443_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, u32, i64, st = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int
        L.fks_build_u64.argtypes = [vp, vp, ctypes.c_int, u64, u64, vp, vp, vp, ctypes.POINTER(vp)]
        L.fks_build_bytes.argtypes = [vp, vp, vp, ctypes.c_int, u64, u64, vp, vp, vp, ctypes.POINTER(vp)]
        L.fks_lookup_u64.argtypes = [vp, vp, u64, vp, vp, i64, vp]
        L.fks_lookup_bytes.argtypes = [vp, vp, vp, u64, vp, vp, i64, vp]
        L.fks_build_batched.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, u32, vp, ctypes.c_int, vp, vp,
                                        vp, ctypes.POINTER(vp), vp]
        L.fks_lookup_batched.argtypes = [vp, vp, vp, vp, vp, u64, vp, vp, i64, vp]
        L.fks_mapset_size.argtypes = [vp]
        L.fks_mapset_size.restype = u32
        L.fks_mapset_get.argtypes = [vp, u32]
        L.fks_mapset_get.restype = vp
        L.fks_map_info.argtypes = [vp, ctypes.POINTER(fks_map_info_t)]
        L.fks_map_export.argtypes = [vp, vp, vp, vp, vp]
        L.fks_map_destroy.argtypes = [vp]
        L.fks_map_destroy.restype = None
        L.fks_mapset_destroy.argtypes = [vp]
        L.fks_mapset_destroy.restype = None
        L.fks_status_str.argtypes = [st]
        L.fks_status_str.restype = ctypes.c_char_p
        L.fks_last_error.argtypes = []
        L.fks_last_error.restype = ctypes.c_char_p
        L.fks_sortmap_build.argtypes = [vp, vp, ctypes.c_int, u64, vp, vp, ctypes.POINTER(vp)]
        L.fks_sortmap_build.restype = st
        L.fks_build_u64_async.argtypes = [vp, vp, ctypes.c_int, u64, u64, vp, vp, vp, ctypes.POINTER(vp)]
        L.fks_build_u64_async.restype = st
        L.fks_build_bytes_async.argtypes = [vp, vp, vp, ctypes.c_int, u64, u64, vp, vp, vp, ctypes.POINTER(vp)]
        L.fks_build_bytes_async.restype = st
        L.fks_build_u64_host.argtypes = [vp, vp, ctypes.c_int, u64, u64, vp, vp, vp, ctypes.POINTER(vp)]
        L.fks_build_u64_host.restype = st
        L.fks_lookup_u64_host.argtypes = [vp, vp, u64, vp, vp, i64, vp]
        L.fks_lookup_u64_host.restype = st
        L.fks_eytzmap_build.argtypes = [vp, vp, ctypes.c_int, u64, vp, vp, ctypes.POINTER(vp)]
        L.fks_eytzmap_build.restype = st
        L.fks_sortmap_lookup.argtypes = [vp, vp, u64, vp, vp, i64, vp]
        L.fks_sortmap_lookup.restype = st
        L.fks_sortmap_export.argtypes = [vp, vp, vp, vp]
        L.fks_sortmap_export.restype = st
        L.fks_sortmap_destroy.argtypes = [vp]
        L.fks_sortmap_destroy.restype = None
        L.fks_profile_enable.argtypes = [ctypes.c_int]
        L.fks_profile_enable.restype = None
        L.fks_last_build_profile.argtypes = [ctypes.POINTER(fks_build_profile)]
        L.fks_last_build_profile.restype = st
        L.fks_kernel_launches.argtypes = []
        L.fks_kernel_launches.restype = u64
        L.fks_test_hold_first_partition.argtypes = [ctypes.c_int]
        L.fks_test_hold_first_partition.restype = None
        L.fks_test_fail_serve_launches.argtypes = [ctypes.c_int]
        L.fks_test_fail_serve_launches.restype = None
        for name in ("fks_build_u64", "fks_build_bytes", "fks_lookup_u64", "fks_lookup_bytes",
                     "fks_build_batched", "fks_lookup_batched", "fks_map_info", "fks_map_export"):
            getattr(L, name).restype = st
        _lib = L
    return _lib


def _check(status: int):
    if status != FKS_OK:
        raise FksError(status, lib().fks_last_error().decode())


def _ptr(t, name="buffer", itemsize=None, numel=None):
    """Device address of a tensor (None passes NULL), after the checks the C
    ABI cannot make on a bare pointer: CUDA memory, dense, of the element
    width the call reads or writes, and at least as long as it needs."""
    if t is None:
        return None
    if not getattr(t, "is_cuda", False):
        raise TypeError(f"{name}: a CUDA tensor is expected")
    if not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is expected")
    if itemsize is not None and t.element_size() != itemsize:
        raise TypeError(f"{name}: elements of {itemsize} bytes are expected, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name}: at least {numel} elements are expected, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _outs(out_vals, out_found, nq: int, value_bytes):
    """Result buffers of a lookup of nq needles: values of the map's width
    (value_bytes() is asked only when values are requested), flags of 1 byte."""
    v = None if out_vals is None else _ptr(out_vals, "out_vals", value_bytes(), nq)
    return v, _ptr(out_found, "out_found", 1, nq)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _val_type(vals) -> int:
    import torch
    if vals.dtype == torch.int64:
        return FKS_VAL_I64
    if vals.dtype == torch.int32:
        return FKS_VAL_I32
    raise TypeError("values must be int32 or int64")


def make_opts(**kw) -> fks_build_opts:
    o = fks_build_opts()
    o.struct_size = ctypes.sizeof(fks_build_opts)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Map:
    """Owning handle of a built map (destroyed with the object)."""

    def __init__(self, handle: int, owner=None, vbytes: int | None = None):
        self.handle = handle
        self._owner = owner  # a MapSet for borrowed handles
        self._vbytes = vbytes  # bytes of a value (4 or 8); asked from the map when unknown

    def info(self) -> fks_map_info_t:
        return fks_map_info(self)

    def value_bytes(self) -> int:
        if self._vbytes is None:
            self._vbytes = 8 if fks_map_info(self).val_type == FKS_VAL_I64 else 4
        return self._vbytes

    def __del__(self):
        if self._owner is None and self.handle and _lib is not None:
            _lib.fks_map_destroy(self.handle)
            self.handle = None


class MapSet:
    def __init__(self, handle: int, status: np.ndarray, owned: bool = True, vbytes: int | None = None):
        self.handle = handle
        self.status = status
        self._owned = owned  # False: the set of a recorded build, freed with it
        self.vbytes = vbytes  # bytes of a value of every map of the set

    def __len__(self):
        return int(lib().fks_mapset_size(self.handle))

    def get(self, j: int):
        h = lib().fks_mapset_get(self.handle, j)
        return Map(h, owner=self, vbytes=self.vbytes) if h else None

    def __del__(self):
        if self._owned and self.handle and _lib is not None:
            _lib.fks_mapset_destroy(self.handle)
            self.handle = None


def fks_build_u64(keys, vals, seed: int, opts: fks_build_opts | None = None, stream=None, alloc=None) -> Map:
    h = ctypes.c_void_p()
    n = keys.numel()
    _check(lib().fks_build_u64(_ptr(keys, "keys", 8), _ptr(vals, "vals", None, n), _val_type(vals), n,
                               seed & (2**64 - 1), ctypes.byref(opts) if opts else None, _aref(alloc),
                               _stream(stream), ctypes.byref(h)))
    return Map(h.value, vbytes=vals.element_size())


def fks_build_u64_async(keys, vals, seed: int, opts: fks_build_opts | None = None, stream=None) -> Map:
    """Start a build and return its handle at once; fks_map_info reports the outcome."""
    h = ctypes.c_void_p()
    _check(lib().fks_build_u64_async(_ptr(keys, "keys", 8), _ptr(vals, "vals", None, keys.numel()),
                                     _val_type(vals), keys.numel(), seed & (2**64 - 1),
                                     ctypes.byref(opts) if opts else None, None, _stream(stream),
                                     ctypes.byref(h)))
    return Map(h.value, vbytes=vals.element_size())


def fks_build_bytes_async(ctx, offs, vals, seed: int, opts: fks_build_opts | None = None, stream=None) -> Map:
    h = ctypes.c_void_p()
    _check(lib().fks_build_bytes_async(_ptr(ctx, "ctx", 1), _ptr(offs, "offs", 8, 1),
                                       _ptr(vals, "vals", None, offs.numel() - 1), _val_type(vals),
                                       offs.numel() - 1, seed & (2**64 - 1), ctypes.byref(opts) if opts else None,
                                       None, _stream(stream), ctypes.byref(h)))
    return Map(h.value, vbytes=vals.element_size())


def fks_map_status(m: Map) -> int:
    """The status fks_map_info returns (waits for an asynchronous build)."""
    info = fks_map_info_t()
    return int(lib().fks_map_info(m.handle, ctypes.byref(info)))


def fks_build_bytes(ctx, offs, vals, seed: int, opts: fks_build_opts | None = None,
                    stream=None, alloc=None) -> Map:
    h = ctypes.c_void_p()
    n = offs.numel() - 1
    _check(lib().fks_build_bytes(_ptr(ctx, "ctx", 1), _ptr(offs, "offs", 8, 1), _ptr(vals, "vals", None, n),
                                 _val_type(vals), n, seed & (2**64 - 1), ctypes.byref(opts) if opts else None,
                                 _aref(alloc), _stream(stream), ctypes.byref(h)))
    return Map(h.value, vbytes=vals.element_size())


def fks_lookup_u64(m: Map, q, out_vals=None, out_found=None, absent: int = -1, stream=None):
    ov, of = _outs(out_vals, out_found, q.numel(), m.value_bytes)
    _check(lib().fks_lookup_u64(m.handle, _ptr(q, "q", 8), q.numel(), ov, of, absent, _stream(stream)))


def _hptr(a, name="buffer", itemsize=None, numel=None):
    """Host address of a CPU tensor or numpy array (None passes NULL), after
    the same checks as _ptr: host memory, dense, element width, length."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        dense, size, count = a.flags.c_contiguous, a.itemsize, a.size
    else:
        if getattr(a, "is_cuda", False):
            raise TypeError(f"{name}: a host buffer is expected")
        dense, size, count = a.is_contiguous(), a.element_size(), a.numel()
    if not dense:
        raise ValueError(f"{name}: a contiguous buffer is expected")
    if itemsize is not None and size != itemsize:
        raise TypeError(f"{name}: elements of {itemsize} bytes are expected")
    if numel is not None and count < numel:
        raise ValueError(f"{name}: at least {numel} elements are expected, got {count}")
    return ctypes.c_void_p(a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())


def _hval_type(v) -> int:
    dt = v.dtype
    if dt in (np.int64, np.dtype(np.int64)) or str(dt) == "torch.int64":
        return FKS_VAL_I64
    if dt in (np.int32, np.dtype(np.int32)) or str(dt) == "torch.int32":
        return FKS_VAL_I32
    raise TypeError(f"values must be int32 or int64, got {dt}")


def fks_build_u64_host(keys, vals, seed: int, opts: fks_build_opts | None = None, stream=None) -> Map:
    """fks_build_u64 over host keys / values (numpy arrays or CPU tensors)."""
    h = ctypes.c_void_p()
    n = len(keys)
    vt = _hval_type(vals)
    _check(lib().fks_build_u64_host(_hptr(keys, "keys", 8), _hptr(vals, "vals", None, n), vt, n, seed & (2**64 - 1),
                                    ctypes.byref(opts) if opts else None, None, _stream(stream), ctypes.byref(h)))
    return Map(h.value, vbytes=8 if vt == FKS_VAL_I64 else 4)


def fks_lookup_u64_host(m: Map, q, out_vals=None, out_found=None, absent: int = -1, stream=None):
    """fks_lookup_u64 over host needles and results; blocks until done."""
    nq = len(q)
    ov = None if out_vals is None else _hptr(out_vals, "out_vals", m.value_bytes(), nq)
    _check(lib().fks_lookup_u64_host(m.handle, _hptr(q, "q", 8), nq, ov, _hptr(out_found, "out_found", 1, nq),
                                     absent, _stream(stream)))


def fks_lookup_bytes(m: Map, qctx, qoffs, out_vals=None, out_found=None, absent: int = -1,
                     stream=None):
    nq = qoffs.numel() - 1
    ov, of = _outs(out_vals, out_found, nq, m.value_bytes)
    _check(lib().fks_lookup_bytes(m.handle, _ptr(qctx, "qctx", 1), _ptr(qoffs, "qoffs", 8, 1), nq, ov, of,
                                  absent, _stream(stream)))


def fks_build_batched(kind: int, keys, ctx, offs, seg: np.ndarray, seeds: np.ndarray, vals,
                      opts: fks_build_opts | None = None, stream=None, raise_on_error=True, alloc=None) -> MapSet:
    if getattr(seg, "is_cuda", False):  # device segment offsets: passed as they are
        m = seg.numel() - 1
        seg_ptr = _ptr(seg, "seg", 8, 1)
        total = None
    else:
        seg = np.ascontiguousarray(seg, np.int64)
        m = seg.size - 1
        seg_ptr = seg.ctypes.data_as(ctypes.c_void_p)
        total = int(seg[-1]) if seg.size else 0
    seeds = np.ascontiguousarray(seeds, np.uint64)
    status = np.zeros(m, np.int32)
    h = ctypes.c_void_p()
    st = lib().fks_build_batched(kind, _ptr(keys, "keys", 8), _ptr(ctx, "ctx", 1), _ptr(offs, "offs", 8),
                                 seg_ptr,
                                 seeds.ctypes.data_as(ctypes.c_void_p), m, _ptr(vals, "vals", None, total),
                                 _val_type(vals), ctypes.byref(opts) if opts else None, _aref(alloc),
                                 _stream(stream), ctypes.byref(h), status.ctypes.data_as(ctypes.c_void_p))
    s = MapSet(h.value, status, vbytes=vals.element_size())
    if raise_on_error or not h.value:
        _check(st)
    return s


def fks_lookup_batched(s: MapSet, map_ids, q=None, qctx=None, qoffs=None, out_vals=None,
                       out_found=None, absent: int = -1, stream=None):
    nq = map_ids.numel()
    ov, of = _outs(out_vals, out_found, nq, lambda: s.vbytes if s.vbytes else 8)
    _check(lib().fks_lookup_batched(s.handle, _ptr(map_ids, "map_ids", 4), _ptr(q, "q", 8, nq),
                                    _ptr(qctx, "qctx", 1), _ptr(qoffs, "qoffs", 8, nq + 1), nq, ov, of, absent,
                                    _stream(stream)))


class BuildGraph:
    """Owning handle of a recorded batched build (fks_build_graph_*).  Keeps
    its input tensors alive: the graph reads them on every run."""

    def __init__(self, handle: int, inputs, m: int):
        self.handle, self._inputs, self.m = handle, inputs, m
        self.status = np.zeros(m, np.int32)

    def mapset(self) -> MapSet:
        """The maps of the last run (owned by the graph)."""
        h = _graph_lib().fks_build_graph_mapset(self.handle)
        vals = self._inputs[3]
        s = MapSet(h, self.status, owned=False, vbytes=vals.element_size())
        s._graph = self  # the graph must outlive the set's use
        return s

    def kernels(self) -> int:
        return int(_graph_lib().fks_build_graph_kernels(self.handle))

    def close(self):
        if self.handle and _lib is not None:
            _lib.fks_build_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def _graph_lib():
    L = lib()
    if not getattr(L, "_graph_types", False):
        vp = ctypes.c_void_p
        L.fks_build_graph_create.argtypes = [ctypes.c_int, vp, vp, vp, vp, ctypes.c_uint32, vp, ctypes.c_int, vp,
                                             vp, vp, ctypes.POINTER(vp)]
        L.fks_build_graph_create.restype = ctypes.c_int
        L.fks_build_graph_run.argtypes = [vp, vp, vp, vp]
        L.fks_build_graph_run.restype = ctypes.c_int
        L.fks_build_graph_mapset.argtypes = [vp]
        L.fks_build_graph_mapset.restype = vp
        L.fks_build_graph_kernels.argtypes = [vp]
        L.fks_build_graph_kernels.restype = ctypes.c_uint32
        L.fks_build_graph_destroy.argtypes = [vp]
        L.fks_build_graph_destroy.restype = None
        L._graph_types = True
    return L


def fks_build_graph_create(kind: int, keys, ctx, offs, seg: np.ndarray, vals,
                           opts: fks_build_opts | None = None, stream=None) -> BuildGraph:
    seg = np.ascontiguousarray(seg, np.int64)
    m = seg.size - 1
    h = ctypes.c_void_p()
    _check(_graph_lib().fks_build_graph_create(kind, _ptr(keys, "keys", 8), _ptr(ctx, "ctx", 1),
                                               _ptr(offs, "offs", 8), seg.ctypes.data_as(ctypes.c_void_p), m,
                                               _ptr(vals, "vals", None, int(seg[-1]) if seg.size else 0),
                                               _val_type(vals), ctypes.byref(opts) if opts else None, None,
                                               _stream(stream), ctypes.byref(h)))
    return BuildGraph(h.value, (keys, ctx, offs, vals), m)


def fks_build_graph_run(g: BuildGraph, seeds: np.ndarray, stream=None, raise_on_error=True) -> np.ndarray:
    """Rebuild every map of the graph with these seeds; per-map statuses."""
    seeds = np.ascontiguousarray(seeds, np.uint64)
    assert seeds.size == g.m
    st = _graph_lib().fks_build_graph_run(g.handle, seeds.ctypes.data_as(ctypes.c_void_p), _stream(stream),
                                          g.status.ctypes.data_as(ctypes.c_void_p))
    if raise_on_error:
        _check(st)
    return g.status.copy()


class fks_tuning(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("key_kind", ctypes.c_uint32),
                ("keys_per_bucket", ctypes.c_uint32), ("thread_search_max", ctypes.c_uint32),
                ("part_ctas_per_sm", ctypes.c_uint32), ("scatter_blocks_per_sm", ctypes.c_uint32),
                ("split_min_keys_log2", ctypes.c_uint32), ("lookup_queries_per_thread", ctypes.c_uint32),
                ("lookup_block", ctypes.c_uint32), ("lookup_blocks_per_sm", ctypes.c_uint32),
                ("tuned", ctypes.c_uint32), ("build_ms", ctypes.c_float), ("lookup_ms", ctypes.c_float),
                ("sample_keys", ctypes.c_uint64), ("part_prefetch", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k not in ("struct_size", "reserved")}


class fks_tune_trial(ctypes.Structure):
    _fields_ = [("param", ctypes.c_uint32), ("value", ctypes.c_uint32), ("ms", ctypes.c_float)]


TUNE_PARAMS = ("thread_search_max", "part_ctas_per_sm", "scatter_blocks_per_sm", "split_min_keys_log2",
               "lookup_queries_per_thread<<16|lookup_block", "lookup_blocks_per_sm", "part_prefetch")


def _tune_lib():
    L = lib()
    if not getattr(L, "_tune_types", False):
        vp = ctypes.c_void_p
        L.fks_autotune.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   vp, ctypes.POINTER(fks_tuning), vp, ctypes.c_uint32,
                                   ctypes.POINTER(ctypes.c_uint32)]
        L.fks_autotune.restype = ctypes.c_int
        L.fks_tuning_get.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(fks_tuning)]
        L.fks_tuning_get.restype = ctypes.c_int
        L.fks_tuning_set.argtypes = [ctypes.POINTER(fks_tuning)]
        L.fks_tuning_set.restype = ctypes.c_int
        L.fks_tuning_reset.argtypes = []
        L.fks_tuning_reset.restype = None
        L._tune_types = True
    return L


def fks_autotune(kind: int = FKS_KEY_U64, keys_per_bucket: int = 1, n: int = 0, nq: int = 0, seed: int = 1,
                 stream=None):
    """Measure the launch shapes on a synthetic sample; (entry, trials)."""
    t = fks_tuning()
    trials = (fks_tune_trial * 256)()
    count = ctypes.c_uint32()
    st = _tune_lib().fks_autotune(kind, keys_per_bucket, n, nq, seed & (2**64 - 1), _stream(stream),
                                  ctypes.byref(t), ctypes.cast(trials, ctypes.c_void_p), 256, ctypes.byref(count))
    if st != FKS_OK:
        raise FksError(st, fks_status_str(st))
    rows = [(TUNE_PARAMS[trials[i].param], trials[i].value, trials[i].ms) for i in range(min(count.value, 256))]
    return t, rows


def fks_tuning_get(kind: int = FKS_KEY_U64, keys_per_bucket: int = 1) -> fks_tuning:
    t = fks_tuning()
    st = _tune_lib().fks_tuning_get(kind, keys_per_bucket, ctypes.byref(t))
    if st != FKS_OK:
        raise FksError(st, fks_status_str(st))
    return t


def fks_tuning_set(t: fks_tuning):
    t.struct_size = ctypes.sizeof(fks_tuning)
    st = _tune_lib().fks_tuning_set(ctypes.byref(t))
    if st != FKS_OK:
        raise FksError(st, fks_status_str(st))


def fks_tuning_reset():
    _tune_lib().fks_tuning_reset()


def fks_tuning_save(path: str):
    L = _tune_lib()
    L.fks_tuning_save.argtypes = [ctypes.c_char_p]
    L.fks_tuning_save.restype = ctypes.c_int
    st = L.fks_tuning_save(path.encode())
    if st != FKS_OK:
        raise FksError(st, f"could not write {path}")


def fks_tuning_load(path: str):
    L = _tune_lib()
    L.fks_tuning_load.argtypes = [ctypes.c_char_p]
    L.fks_tuning_load.restype = ctypes.c_int
    st = L.fks_tuning_load(path.encode())
    if st != FKS_OK:
        raise FksError(st, f"could not read a tuning table from {path}")


def fks_build_u64_noalloc(keys, vals, seed: int, desc_out, slots_out,
                          opts: fks_build_opts | None = None, stream=None) -> fks_map_info_t:
    """The allocation-free build: the caller owns every output buffer
    (desc_out int64[n], slots_out int64[2 * capacity]); scratch comes from a
    fixed array inside the library (n <= 262144)."""
    f = lib().fks_build_u64_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                  ctypes.POINTER(fks_map_info_t), ctypes.c_void_p]
    f.restype = ctypes.c_int
    info = fks_map_info_t()
    st = f(_ptr(keys, "keys", 8), _ptr(vals, "vals", None, keys.numel()), _val_type(vals), keys.numel(),
           seed & (2**64 - 1), ctypes.byref(opts) if opts else None, _ptr(desc_out, "desc_out", 8),
           _ptr(slots_out, "slots_out", 8),
           slots_out.numel() // 2, ctypes.byref(info), _stream(stream))
    if st != FKS_OK:
        raise FksError(st, fks_status_str(st))
    return info


def fks_map_info(m: Map) -> fks_map_info_t:
    info = fks_map_info_t()
    _check(lib().fks_map_info(m.handle, ctypes.byref(info)))
    return info


def fks_map_export(m: Map, stream=None):
    """(desc uint64[buckets], slots uint64[S, 2 or 4], ctx uint8[] or None) on the host."""
    info = fks_map_info(m)
    words = 4 if info.key_kind == FKS_KEY_BYTES else 2
    desc = np.empty(info.buckets, np.uint64)
    slots = np.empty((info.slots, words), np.uint64)
    ctx = np.empty(max(info.context_bytes, 1), np.uint8) if info.key_kind == FKS_KEY_BYTES else None
    _check(lib().fks_map_export(m.handle, desc.ctypes.data_as(ctypes.c_void_p),
                                slots.ctypes.data_as(ctypes.c_void_p),
                                None if ctx is None else ctx.ctypes.data_as(ctypes.c_void_p),
                                _stream(stream)))
    if ctx is not None:
        ctx = ctx[: info.context_bytes]
    return desc, slots, ctx


def fks_map_export_records(m: Map, stream=None) -> np.ndarray:
    """The inline-singleton records, uint64[buckets, 2], on the host."""
    info = fks_map_info(m)
    rec = np.empty((info.buckets, 2), np.uint64)
    L = lib()
    L.fks_map_export_records.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.fks_map_export_records.restype = ctypes.c_int
    _check(L.fks_map_export_records(m.handle, rec.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return rec


def fks_map_import(info: fks_map_info_t, desc: np.ndarray, slots: np.ndarray, ctx=None, stream=None) -> Map:
    """A map from exported tables (host arrays as fks_map_export returns them)."""
    L = lib()
    L.fks_map_import.argtypes = [ctypes.POINTER(fks_map_info_t), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    L.fks_map_import.restype = ctypes.c_int
    desc = np.ascontiguousarray(desc, np.uint64)
    slots = np.ascontiguousarray(slots, np.uint64)
    cptr = None
    if ctx is not None:
        ctx = np.ascontiguousarray(ctx, np.uint8)
        cptr = ctx.ctypes.data_as(ctypes.c_void_p) if ctx.size else ctypes.c_void_p(np.zeros(1, np.uint8).ctypes.data)
    h = ctypes.c_void_p()
    _check(L.fks_map_import(ctypes.byref(info), desc.ctypes.data_as(ctypes.c_void_p),
                            slots.ctypes.data_as(ctypes.c_void_p), cptr, None, _stream(stream), ctypes.byref(h)))
    return Map(h.value, vbytes=8 if info.val_type == FKS_VAL_I64 else 4)


def fks_map_save(m: Map, path: str, stream=None):
    """Checkpoint a map: its tables and metadata into one .npz file."""
    info = fks_map_info(m)
    desc, slots, ctx = fks_map_export(m, stream)
    meta = np.array([getattr(info, k) for k, _ in fks_map_info_t._fields_], np.uint64)
    np.savez(path, meta=meta, desc=desc, slots=slots, ctx=ctx if ctx is not None else np.zeros(0, np.uint8))


def fks_map_load(path: str, stream=None) -> Map:
    """Resume a map saved by fks_map_save."""
    z = np.load(path)
    info = fks_map_info_t()
    for (k, _), v in zip(fks_map_info_t._fields_, z["meta"].tolist()):
        setattr(info, k, int(v))
    ctx = z["ctx"] if info.key_kind == FKS_KEY_BYTES else None
    return fks_map_import(info, z["desc"], z["slots"], ctx, stream)


class SortMap:
    """Owning handle of a sorted-array map (the search-based comparison)."""

    def __init__(self, handle: int, n: int, vbytes: int = 8):
        self.handle, self.n, self.vbytes = handle, n, vbytes

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.fks_sortmap_destroy(self.handle)
            self.handle = None


def fks_sortmap_build(keys, vals, stream=None) -> SortMap:
    h = ctypes.c_void_p()
    _check(lib().fks_sortmap_build(_ptr(keys, "keys", 8), _ptr(vals, "vals", None, keys.numel()),
                                   _val_type(vals), keys.numel(), None, _stream(stream), ctypes.byref(h)))
    return SortMap(h.value, keys.numel(), vals.element_size())


def fks_eytzmap_build(keys, vals, stream=None) -> SortMap:
    h = ctypes.c_void_p()
    _check(lib().fks_eytzmap_build(_ptr(keys, "keys", 8), _ptr(vals, "vals", None, keys.numel()),
                                   _val_type(vals), keys.numel(), None, _stream(stream), ctypes.byref(h)))
    return SortMap(h.value, keys.numel(), vals.element_size())


def fks_sortmap_lookup(m: SortMap, q, out_vals=None, out_found=None, absent: int = -1, stream=None):
    ov, of = _outs(out_vals, out_found, q.numel(), lambda: m.vbytes)
    _check(lib().fks_sortmap_lookup(m.handle, _ptr(q, "q", 8), q.numel(), ov, of, absent, _stream(stream)))


def fks_sortmap_export(m: SortMap, stream=None):
    k = np.empty(m.n, np.uint64)
    v = np.empty(m.n, np.int64)
    _check(lib().fks_sortmap_export(m.handle, k.ctypes.data_as(ctypes.c_void_p),
                                    v.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return k, v


# ------------------------------------------------------------------ serving
FKS_SERVE_BATCHED, FKS_SERVE_PER_CALL = 0, 1
FKS_REQ_BUILD, FKS_REQ_LOOKUP = 0, 1


class fks_server_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("memory_budget", ctypes.c_uint64),
                ("max_maps", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("build_workers", ctypes.c_uint32), ("max_batch_requests", ctypes.c_uint32),
                ("max_inflight_batches", ctypes.c_uint32)]


class fks_request(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("type", ctypes.c_uint32), ("map_id", ctypes.c_uint32),
                ("key_kind", ctypes.c_uint32), ("val_type", ctypes.c_uint32),
                ("keys", ctypes.c_void_p), ("ctx", ctypes.c_void_p), ("offs", ctypes.c_void_p),
                ("ctx_bytes", ctypes.c_uint64), ("vals", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("q", ctypes.c_void_p), ("qctx", ctypes.c_void_p),
                ("qoffs", ctypes.c_void_p), ("nq", ctypes.c_uint64), ("out_vals", ctypes.c_void_p),
                ("out_found", ctypes.c_void_p), ("absent", ctypes.c_int64)]


class fks_server_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "builds", "lookups", "queries",
                                                 "batches", "evictions", "rejected", "resident_bytes",
                                                 "peak_resident_bytes")] + \
               [(k, ctypes.c_double) for k in ("span_s", "p50_us", "p99_us", "p999_us", "lookup_p50_us",
                                                 "lookup_p99_us", "build_p50_us", "build_p99_us")]


def _server_lib():
    L = lib()
    if not getattr(L, "_server_types", False):
        vp, u64 = ctypes.c_void_p, ctypes.c_uint64
        L.fks_server_create.argtypes = [ctypes.POINTER(fks_server_opts), ctypes.POINTER(vp)]
        L.fks_server_create.restype = ctypes.c_int
        L.fks_server_submit.argtypes = [vp, ctypes.POINTER(fks_request), ctypes.POINTER(u64)]
        L.fks_server_submit.restype = ctypes.c_int
        L.fks_server_replay.argtypes = [vp, vp, vp, u64, vp]
        L.fks_server_replay.restype = ctypes.c_int
        L.fks_server_wait.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.fks_server_wait.restype = ctypes.c_int
        L.fks_server_drain.argtypes = [vp]
        L.fks_server_drain.restype = ctypes.c_int
        L.fks_server_stats.argtypes = [vp, ctypes.POINTER(fks_server_stats_t)]
        L.fks_server_stats.restype = ctypes.c_int
        L.fks_server_map.argtypes = [vp, ctypes.c_uint32]
        L.fks_server_map.restype = vp
        L.fks_server_destroy.argtypes = [vp]
        L.fks_server_destroy.restype = None
        L._server_types = True
    return L


class Server:
    """Owning handle of a serving loop (fks_server_*)."""

    def __init__(self, handle: int):
        self.handle = handle

    def close(self):
        if self.handle and _lib is not None:
            _lib.fks_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def fks_server_create(memory_budget: int, max_maps: int, mode: int = FKS_SERVE_BATCHED,
                      build_workers: int = 0, max_batch_requests: int = 0,
                      max_inflight_batches: int = 0) -> Server:
    o = fks_server_opts(ctypes.sizeof(fks_server_opts), memory_budget, max_maps, mode, build_workers,
                        max_batch_requests, max_inflight_batches)
    h = ctypes.c_void_p()
    _check(_server_lib().fks_server_create(ctypes.byref(o), ctypes.byref(h)))
    return Server(h.value)


def make_request(**kw) -> fks_request:
    r = fks_request()
    r.struct_size = ctypes.sizeof(fks_request)
    for k, v in kw.items():
        setattr(r, k, v)
    return r


def fks_server_submit(s: Server, req: fks_request) -> int:
    t = ctypes.c_uint64()
    _check(_server_lib().fks_server_submit(s.handle, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def fks_server_replay(s: Server, reqs, arrival_us: np.ndarray) -> np.ndarray:
    """reqs: a ctypes array of fks_request; returns the tickets."""
    arr = np.ascontiguousarray(arrival_us, np.float64)
    tickets = np.zeros(arr.size, np.uint64)
    _check(_server_lib().fks_server_replay(s.handle, ctypes.cast(reqs, ctypes.c_void_p),
                                           arr.ctypes.data_as(ctypes.c_void_p), arr.size,
                                           tickets.ctypes.data_as(ctypes.c_void_p)))
    return tickets


def fks_server_wait(s: Server, ticket: int):
    st, lat = ctypes.c_int(), ctypes.c_double()
    _check(_server_lib().fks_server_wait(s.handle, ticket, ctypes.byref(st), ctypes.byref(lat)))
    return st.value, lat.value


def fks_server_drain(s: Server):
    _check(_server_lib().fks_server_drain(s.handle))


def fks_server_stats(s: Server) -> fks_server_stats_t:
    o = fks_server_stats_t()
    _check(_server_lib().fks_server_stats(s.handle, ctypes.byref(o)))
    return o


def fks_server_map(s: Server, map_id: int):
    h = _server_lib().fks_server_map(s.handle, map_id)
    return Map(h, owner=s) if h else None


def fks_status_str(status: int) -> str:
    return lib().fks_status_str(status).decode()


def fks_profile_enable(on: bool):
    lib().fks_profile_enable(1 if on else 0)


def fks_last_build_profile() -> fks_build_profile:
    p = fks_build_profile()
    _check(lib().fks_last_build_profile(ctypes.byref(p)))
    return p


def fks_kernel_launches() -> int:
    return int(lib().fks_kernel_launches())


def fks_test_hold_first_partition(on: bool):
    lib().fks_test_hold_first_partition(1 if on else 0)


def fks_test_fail_serve_launches(n: int):
    lib().fks_test_fail_serve_launches(int(n))
