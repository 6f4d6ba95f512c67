"""The serving loop: continuous batching over resident maps under a memory
budget.  Every result must be the same served in the mix as alone (integer
results: exactly), admission evicts least-recently-used maps, and a request
that does not fit is denied."""
import numpy as np
import pytest

from paper_2508_11443_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch  # noqa: F401
    from paper_2508_11443_b300 import build, fks
    build.build()
    return fks


@pytest.fixture(scope="module")
def strings():
    return W.string_workload(1 << 14, 1 << 14, 0.0, seed=21)


def small_plan(strings, n_req, seed, budget):
    return W.serving_plan(n_req, seed, budget, strings.offs, prefill=8, u64_n=(2**10, 2**14),
                          str_n=(2**10, 2**12), nq_range=(1, 2**12), u64_pool=2**16)


def run(F, data, mode, rate=2e5):
    import torch
    P = data.plan
    srv = F.fks_server_create(memory_budget=P.budget, max_maps=int(P.map_id.max()) + 1, mode=mode,
                              max_batch_requests=64)
    arr = W.poisson_arrivals_us(P.kind.size, rate, 3)
    tickets = F.fks_server_replay(srv, data.reqs, arr)
    F.fks_server_drain(srv)
    res = [F.fks_server_wait(srv, int(t)) for t in tickets]
    st = F.fks_server_stats(srv)
    torch.cuda.synchronize()
    return srv, res, st, data.out.cpu().numpy().copy(), data.found.cpu().numpy().copy()


def expected(data):
    P = data.plan
    exp_f = np.zeros(data.out.numel(), np.uint8)
    exp_v = np.full(data.out.numel(), -1, np.int64)
    ue, se = data.u_expect.cpu().numpy(), data.s_expect.cpu().numpy()
    for r in np.nonzero(P.kind == 1)[0]:
        a, nq = int(data.out_start[r]), int(P.nq[r])
        if P.key_kind[r] == 0:
            e = ue[data.u_start[data.u_index[r]]:data.u_start[data.u_index[r]] + nq]
        else:
            e = se[data.s_start[data.s_index[r]]:data.s_start[data.s_index[r]] + nq]
        exp_v[a:a + nq] = e
        exp_f[a:a + nq] = (e >= 0)
    return exp_v, exp_f


def test_served_results_are_correct_and_equal_per_call(F, strings):
    P = small_plan(strings, 400, seed=5, budget=6 << 20)
    data = W.ServeData(P, seed=9, u64_pool=2**16, strings=strings)
    exp_v, exp_f = expected(data)
    srv, res, st, out_b, found_b = run(F, data, F.FKS_SERVE_BATCHED)
    assert all(s == F.FKS_OK for s, _ in res), [s for s, _ in res if s]
    assert st.evictions > 0 and st.batches < st.lookups
    assert np.array_equal(found_b, exp_f) and np.array_equal(out_b, exp_v)
    srv.close()
    data.out.fill_(7)
    data.found.fill_(7)
    srv2, res2, st2, out_p, found_p = run(F, data, F.FKS_SERVE_PER_CALL)
    assert all(s == F.FKS_OK for s, _ in res2)
    assert st2.batches == 0
    assert np.array_equal(out_p, out_b) and np.array_equal(found_p, found_b)
    srv2.close()


def test_a_served_lookup_equals_the_same_lookup_alone(F, strings):
    import torch
    P = small_plan(strings, 200, seed=6, budget=64 << 20)
    data = W.ServeData(P, seed=10, u64_pool=2**16, strings=strings)
    srv, res, st, out_b, found_b = run(F, data, F.FKS_SERVE_BATCHED)
    looks = np.nonzero(P.kind == 1)[0][:25]
    for r in looks:
        req = data.reqs[r]
        m = F.fks_server_map(srv, int(P.map_id[r]))
        assert m is not None
        nq = int(P.nq[r])
        out = torch.empty(nq, dtype=torch.int64, device="cuda")
        found = torch.empty(nq, dtype=torch.uint8, device="cuda")
        import ctypes
        if P.key_kind[r] == 0:
            st_ = F.lib().fks_lookup_u64(m.handle, ctypes.c_void_p(req.q), nq, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(found.data_ptr()), -1, None)
        else:
            st_ = F.lib().fks_lookup_bytes(m.handle, ctypes.c_void_p(req.qctx), ctypes.c_void_p(req.qoffs), nq,
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(found.data_ptr()), -1,
                                          None)
        assert st_ == F.FKS_OK
        torch.cuda.synchronize()
        a = int(data.out_start[r])
        assert np.array_equal(found.cpu().numpy(), found_b[a:a + nq])
        assert np.array_equal(out.cpu().numpy().astype(np.int64), out_b[a:a + nq])
    srv.close()


def test_lru_eviction_admission_and_parked_lookups(F):
    import torch
    keys = [torch.from_numpy(W.key_stream(100 + i, 1000).view(np.int64)).cuda() for i in range(5)]
    vals = torch.arange(1000, dtype=torch.int64, device="cuda")
    out = torch.empty(1000, dtype=torch.int64, device="cuda")
    found = torch.empty(1000, dtype=torch.uint8, device="cuda")
    srv = F.fks_server_create(memory_budget=150_000, max_maps=8)  # two maps of 72 000 B fit

    def build(i):
        return F.fks_server_submit(srv, F.make_request(type=F.FKS_REQ_BUILD, map_id=i, key_kind=0,
                                                       val_type=F.FKS_VAL_I64, keys=keys[i].data_ptr(),
                                                       vals=vals.data_ptr(), n=1000, seed=i))

    def lookup(i, k):
        return F.fks_server_submit(srv, F.make_request(type=F.FKS_REQ_LOOKUP, map_id=i, key_kind=0,
                                                       q=keys[k].data_ptr(), nq=1000, out_vals=out.data_ptr(),
                                                       out_found=found.data_ptr(), absent=-1))

    t0 = build(0)
    tl = lookup(0, 0)           # parked until map 0 is built
    assert F.fks_server_wait(srv, tl)[0] == F.FKS_OK
    torch.cuda.synchronize()
    assert found.cpu().numpy().all() and np.array_equal(out.cpu().numpy(), np.arange(1000))
    assert F.fks_server_wait(srv, t0)[0] == F.FKS_OK
    build(1)
    F.fks_server_wait(srv, lookup(0, 0))          # map 0 is now the most recently used
    F.fks_server_wait(srv, build(2))              # evicts map 1 (least recently used)
    assert F.fks_server_wait(srv, lookup(1, 1))[0] == F.FKS_ERR_EVICTED
    assert F.fks_server_wait(srv, lookup(0, 0))[0] == F.FKS_OK
    assert F.fks_server_wait(srv, lookup(2, 2))[0] == F.FKS_OK
    st = F.fks_server_stats(srv)
    assert st.evictions == 1 and st.resident_bytes == 144_000
    # a map larger than the whole budget is denied
    big = torch.from_numpy(W.key_stream(7, 3000).view(np.int64)).cuda()
    bv = torch.arange(3000, dtype=torch.int64, device="cuda")
    t = F.fks_server_submit(srv, F.make_request(type=F.FKS_REQ_BUILD, map_id=5, key_kind=0, val_type=F.FKS_VAL_I64,
                                                keys=big.data_ptr(), vals=bv.data_ptr(), n=3000, seed=1))
    assert F.fks_server_wait(srv, t)[0] == F.FKS_ERR_OUT_OF_MEMORY
    assert F.fks_server_stats(srv).rejected == 1
    srv.close()


def test_a_failed_batch_launch_fails_its_requests_only(F):
    """A lookup batch whose launch fails (injected on the host: the launch is
    not issued and reports a launch error) completes each of its requests
    with FKS_ERR_CUDA; the server, the context and the next batches are
    unaffected."""
    import torch
    keys = torch.from_numpy(W.key_stream(300, 5000).view(np.int64)).cuda()
    vals = torch.arange(5000, dtype=torch.int64, device="cuda")
    out = torch.full((5000,), 7, dtype=torch.int64, device="cuda")
    found = torch.zeros(5000, dtype=torch.uint8, device="cuda")
    srv = F.fks_server_create(memory_budget=1 << 30, max_maps=2)
    try:
        t = F.fks_server_submit(srv, F.make_request(type=F.FKS_REQ_BUILD, map_id=0, key_kind=0,
                                                    val_type=F.FKS_VAL_I64, keys=keys.data_ptr(),
                                                    vals=vals.data_ptr(), n=5000, seed=3))
        assert F.fks_server_wait(srv, t)[0] == F.FKS_OK

        def lookup():
            return F.fks_server_submit(srv, F.make_request(type=F.FKS_REQ_LOOKUP, map_id=0, key_kind=0,
                                                           q=keys.data_ptr(), nq=5000, out_vals=out.data_ptr(),
                                                           out_found=found.data_ptr(), absent=-1))

        F.fks_test_fail_serve_launches(1)
        assert F.fks_server_wait(srv, lookup())[0] == F.FKS_ERR_CUDA
        torch.cuda.synchronize()
        assert (out.cpu().numpy() == 7).all() and not found.cpu().numpy().any()  # nothing was written
        assert F.fks_server_wait(srv, lookup())[0] == F.FKS_OK
        torch.cuda.synchronize()
        assert found.cpu().numpy().all() and np.array_equal(out.cpu().numpy(), np.arange(5000))
    finally:
        F.fks_test_fail_serve_launches(0)
        srv.close()
