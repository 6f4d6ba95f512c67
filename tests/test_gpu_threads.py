"""Host threads that build and query maps at the same time, each on its own
stream (the library keeps per-thread staging buffers and one process-wide
tuning table): every thread's tables equal the oracle's and its lookups the
workload's truth, as when run alone."""
import threading

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


def test_concurrent_builds_and_lookups(F):
    import torch
    cases = [(W.u64_workload(n, 30000, 0.6, seed=100 + i), 11 + i, lam)
             for i, (n, lam) in enumerate([(70001, 1), (1 << 20, 1), (123457, 4), (3000, 16), ((1 << 20) + 3, 2),
                                           (50000, 8)])]
    expect = [O.build_u64(w.keys, w.vals, seed=seed, keys_per_bucket=lam) for w, seed, lam in cases]
    results = [None] * len(cases)
    errors = []
    barrier = threading.Barrier(len(cases))

    def worker(i):
        try:
            torch.cuda.set_device(0)
            w, seed, lam = cases[i]
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                keys = torch.from_numpy(w.keys.view(np.int64)).cuda()
                vals = torch.from_numpy(w.vals).cuda()
                q = torch.from_numpy(w.queries.view(np.int64)).cuda()
                out = torch.empty(len(w.queries), dtype=torch.int64, device="cuda")
                found = torch.empty(len(w.queries), dtype=torch.uint8, device="cuda")
                stream.synchronize()
                barrier.wait()
                for rep in range(3):  # builds and lookups of all threads interleave
                    m = F.fks_build_u64(keys, vals, seed, opts=F.make_opts(keys_per_bucket=lam), stream=stream)
                    F.fks_lookup_u64(m, q, out, found, -1, stream=stream)
                    stream.synchronize()
                d, s, _ = F.fks_map_export(m, stream=stream)
                results[i] = (d, s, out.cpu().numpy(), found.cpu().numpy())
        except Exception as e:  # reported by the main thread
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for (w, seed, lam), om, (d, s, out, found) in zip(cases, expect, results):
        assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots)
        assert np.array_equal(found, w.expect_found)
        assert np.array_equal(out, np.where(w.expect_found == 1, w.expect_vals, -1))


def test_concurrent_async_builds(F):
    import torch
    ws = [W.u64_workload(n, 100, 0.5, seed=200 + n) for n in (5000, 300000, 77777, (1 << 20) + 1)]
    keys = [torch.from_numpy(w.keys.view(np.int64)).cuda() for w in ws]
    vals = [torch.from_numpy(w.vals).cuda() for w in ws]
    torch.cuda.synchronize()
    maps = [F.fks_build_u64_async(k, v, 9) for k, v in zip(keys, vals)]  # all in flight at once
    for w, m in zip(ws, maps):
        assert F.fks_map_status(m) == F.FKS_OK
        d, s, _ = F.fks_map_export(m)
        om = O.build_u64(w.keys, w.vals, seed=9)
        assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots)


FIRST_USE = r"""
import sys, threading
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import oracle as O
from paper_2508_11443_b300 import fks as F, workloads as W

torch.cuda.set_device(0)
torch.zeros(1, device="cuda")
# u64 maps above and below the two-level grouping size, and string maps: the
# first calls into the library in this process, from four threads at once
cases = [("u", W.u64_workload((1 << 20) + 5, 1, 1.0, seed=31), 3), ("u", W.u64_workload(40000, 1, 1.0, seed=32), 4),
         ("s", W.string_workload(1 << 20, 1, 1.0, seed=33), 5), ("s", W.string_workload(30000, 1, 1.0, seed=34), 6)]
barrier = threading.Barrier(len(cases))
got, errors = [None] * len(cases), []

def run(i):
    try:
        kind, w, seed = cases[i]
        torch.cuda.set_device(0)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            if kind == "u":
                k = torch.from_numpy(w.keys.view(np.int64)).cuda()
                v = torch.from_numpy(w.vals).cuda()
                s.synchronize()
                barrier.wait()
                m = F.fks_build_u64(k, v, seed)
            else:
                c, o = torch.from_numpy(w.ctx).cuda(), torch.from_numpy(w.offs).cuda()
                v = torch.from_numpy(w.vals).cuda()
                s.synchronize()
                barrier.wait()
                m = F.fks_build_bytes(c, o, v, seed)
            got[i] = F.fks_map_export(m)[:2]
    except Exception as e:  # reported by the parent
        errors.append(repr(e))

ts = [threading.Thread(target=run, args=(i,)) for i in range(len(cases))]
for t in ts:
    t.start()
for t in ts:
    t.join()
assert not errors, errors
for (kind, w, seed), (d, sl) in zip(cases, got):
    om = O.build_u64(w.keys, w.vals, seed=seed) if kind == "u" else O.build_bytes(w.ctx, w.offs, w.vals, seed=seed)
    assert np.array_equal(d, om.desc) and np.array_equal(sl, om.slots), kind
print("first use ok")
"""


def test_concurrent_first_use_in_a_fresh_process(F):
    """The library's one-time set-up (kernel attributes, occupancy, the SM
    count) happens under concurrent first calls: four threads of a fresh
    process start their builds together as the process's first calls into
    the library, and every table equals the oracle's."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", FIRST_USE, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "first use ok" in r.stdout
