"""fks_build_u64_noalloc, the uint64 build for callers that cannot allocate
device memory: a service whose whole device memory belongs to its own pool or
budget, or a loop that cannot pay for cudaMalloc / cudaFree (which may
synchronise the device).  Such a caller hands in the inputs and the output
tables; the library takes its scratch from one fixed array compiled into it.

The tables it writes must be byte-for-byte those of the allocating
fks_build_u64 (integer tables: the tolerance is zero), on consecutive calls
that reuse the same scratch array.  This file runs last in the suite so that
a failure here never hides the others; it also passes alone in a fresh
process, where its first call is the library's first use of the device."""
import ctypes

import numpy as np
import pytest

from paper_2508_11443_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _entry(fks):
    f = fks.lib().fks_build_u64_noalloc
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    f.argtypes = [vp, vp, ctypes.c_int, u64, u64, vp, vp, vp, u64,
                  ctypes.POINTER(fks.fks_map_info_t), vp]
    f.restype = ctypes.c_int
    return f


def test_noalloc_build_equals_allocating_build_on_consecutive_calls():
    import torch
    from paper_2508_11443_b300 import build, fks
    build.build()
    f = _entry(fks)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # a larger map, then a smaller one: stale scratch contents must not leak
    for n, seed in ((200_000, 5), (3_001, 9)):
        w = W.u64_workload(n, 1, 0.5, seed=n)
        keys = torch.from_numpy(w.keys.view(np.int64)).cuda()
        vals = torch.from_numpy(w.vals).cuda()
        cap = 4 * n
        desc = torch.full((n,), -7, dtype=torch.int64, device="cuda")
        slots = torch.full((2 * cap,), -7, dtype=torch.int64, device="cuda")
        info = fks.fks_map_info_t()
        st = f(keys.data_ptr(), vals.data_ptr(), fks.FKS_VAL_I64, n, seed, None, desc.data_ptr(),
               slots.data_ptr(), cap, ctypes.byref(info), stream)
        torch.cuda.synchronize()
        assert st == fks.FKS_OK, fks.fks_status_str(st)
        ref = fks.fks_build_u64(keys, vals, seed)
        rdesc, rslots, _ = fks.fks_map_export(ref)
        rinfo = fks.fks_map_info(ref)
        assert (info.slots, info.round) == (rinfo.slots, rinfo.round)
        assert np.array_equal(desc.cpu().numpy().view(np.uint64), rdesc)
        got = slots.cpu().numpy().view(np.uint64)[: 2 * info.slots].reshape(-1, 2)
        assert np.array_equal(got, rslots)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    from paper_2508_11443_b300 import build, fks
    build.build()
    f = _entry(fks)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = 262144 + 1  # FKS_NOALLOC_MAX_KEYS + 1
    keys = torch.zeros(n, dtype=torch.int64, device="cuda")
    vals = torch.zeros(n, dtype=torch.int64, device="cuda")
    desc = torch.empty(n, dtype=torch.int64, device="cuda")
    slots = torch.empty(8 * n, dtype=torch.int64, device="cuda")
    st = f(keys.data_ptr(), vals.data_ptr(), fks.FKS_VAL_I64, n, 1, None, desc.data_ptr(),
           slots.data_ptr(), 4 * n, None, stream)
    assert st == fks.FKS_ERR_INVALID_ARG
    # too small an output table is rejected too
    st = f(keys.data_ptr(), vals.data_ptr(), fks.FKS_VAL_I64, 1000, 1, None, desc.data_ptr(),
           slots.data_ptr(), 3999, None, stream)
    assert st == fks.FKS_ERR_INVALID_ARG
