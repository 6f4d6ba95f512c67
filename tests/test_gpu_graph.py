"""Recorded batched builds (fks_build_graph_*): the first pass of a batched
build recorded once as a CUDA graph and replayed.  Every run's tables equal the
oracle's and fks_build_batched's, byte for byte; a run reads the bound buffers'
current contents and the run's seeds; maps that must redraw finish through the
ordinary pass loop; the two-level grouping of large passes replays too."""
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


def tables(F, S, j):
    d, s, _ = F.fks_map_export(S.get(j))
    return d, s


def check_u64_maps(F, S, keys, vals, seg, seeds, maps, **opts):
    for j in maps:
        k = keys[seg[j]:seg[j + 1]]
        v = vals[seg[j]:seg[j + 1]]
        om = O.build_u64(k, v, seed=int(seeds[j]), **opts)
        d, s = tables(F, S, j)
        assert np.array_equal(d, om.desc) and np.array_equal(s, om.slots), j


def batched_lookup(F, S, ids, q):
    import torch
    out = torch.empty(len(q), dtype=torch.int64, device="cuda")
    found = torch.empty(len(q), dtype=torch.uint8, device="cuda")
    F.fks_lookup_batched(S, dev(ids.astype(np.uint32)), q=dev(q), out_vals=out, out_found=found)
    torch.cuda.synchronize()
    return out.cpu().numpy(), found.cpu().numpy()


def test_graph_runs_equal_oracle_and_batched(F):
    import torch
    b = W.batched_workload(64, 16, 1 << 14, 20000, 0.75, seed=21)
    keys_d, vals_d = dev(b.keys), dev(b.vals)
    g = F.fks_build_graph_create(F.FKS_KEY_U64, keys_d, None, None, b.seg_offs, vals_d)
    assert g.kernels() >= 4
    before = F.fks_kernel_launches()
    st = F.fks_build_graph_run(g, b.seeds)
    assert (st == 0).all()
    assert F.fks_kernel_launches() - before >= g.kernels()
    S = g.mapset()
    assert len(S) == 64
    check_u64_maps(F, S, b.keys, b.vals, b.seg_offs, b.seeds, range(64))
    B = F.fks_build_batched(F.FKS_KEY_U64, keys_d, None, None, b.seg_offs, b.seeds, vals_d)
    for j in range(0, 64, 5):
        d, s = tables(F, S, j)
        d2, s2 = tables(F, B, j)
        assert np.array_equal(d, d2) and np.array_equal(s, s2)
    out, found = batched_lookup(F, S, b.q_map, b.q_keys)
    assert np.array_equal(found, b.expect_found)
    assert np.array_equal(out, np.where(b.expect_found == 1, b.expect_vals, -1))
    # second run: new contents of the same buffers (other keys, same segment
    # sizes) and new seeds
    fresh = W.key_stream(977, b.keys.size)
    keys_d.copy_(dev(fresh))
    vals2 = (b.vals * 3 + 1).astype(np.int64)
    vals_d.copy_(dev(vals2))
    seeds2 = b.seeds + np.uint64(1000)
    st = F.fks_build_graph_run(g, seeds2)
    assert (st == 0).all()
    check_u64_maps(F, S, fresh, vals2, b.seg_offs, seeds2, range(0, 64, 3))
    del S, B
    g.close()
    torch.cuda.synchronize()


def test_graph_maps_that_redraw_finish_in_the_pass_loop(F):
    """bound_factor 2 (S <= 2n, while E[S] = 2n - 1) sends a large share of the
    maps to a second level-one round; the tables still equal the oracle's."""
    b = W.batched_workload(40, 64, 4096, 100, 0.75, seed=33)
    opts = F.make_opts(bound_factor=2)
    g = F.fks_build_graph_create(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, dev(b.vals), opts=opts)
    for rep in range(2):
        seeds = b.seeds + np.uint64(17 * rep)
        st = F.fks_build_graph_run(g, seeds)
        assert (st == 0).all()
        S = g.mapset()
        rounds = [F.fks_map_info(S.get(j)).round for j in range(40)]
        assert max(rounds) >= 1  # some maps redrew
        check_u64_maps(F, S, b.keys, b.vals, b.seg_offs, seeds, range(40), bound_factor=2)
    g.close()


def test_graph_two_level_grouping(F):
    """A pass of more than 2^20 keys groups them in two radix levels; the
    recorded pass replays those kernels too."""
    b = W.batched_workload(24, 1 << 15, 1 << 17, 1 << 16, 0.75, seed=41)
    assert b.seg_offs[-1] >= (1 << 20)
    g = F.fks_build_graph_create(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, dev(b.vals))
    assert g.kernels() >= 10  # the split kernels are in the graph
    st = F.fks_build_graph_run(g, b.seeds)
    assert (st == 0).all()
    S = g.mapset()
    check_u64_maps(F, S, b.keys, b.vals, b.seg_offs, b.seeds, [0, 7, 23])
    out, found = batched_lookup(F, S, b.q_map, b.q_keys)
    assert np.array_equal(found, b.expect_found)
    assert np.array_equal(out, np.where(b.expect_found == 1, b.expect_vals, -1))
    g.close()


def test_graph_strings(F):
    parts = [W.string_workload(n, 10, 0.5, seed=60 + n) for n in (5, 900, 1, 3000)]
    ctx = np.concatenate([p.ctx for p in parts])
    offs = [np.zeros(1, np.int64)]
    base = 0
    for p in parts:
        offs.append(p.offs[1:] + base)
        base += p.offs[-1]
    offs = np.concatenate(offs)
    seg = np.cumsum([0] + [p.offs.size - 1 for p in parts])
    vals = np.concatenate([p.vals for p in parts]).astype(np.int32)
    g = F.fks_build_graph_create(F.FKS_KEY_BYTES, None, dev(ctx), dev(offs), seg, dev(vals))
    for rep in range(2):
        seeds = np.array([21, 22, 23, 24], np.uint64) + np.uint64(rep)
        st = F.fks_build_graph_run(g, seeds)
        assert (st == 0).all()
        S = g.mapset()
        for j, p in enumerate(parts):
            om = O.build_bytes(p.ctx, p.offs, p.vals, seed=int(seeds[j]))
            d, s = tables(F, S, j)
            exp = om.slots.copy()
            exp[:, 1] += np.uint64(offs[seg[j]])  # offsets into the set's shared context
            assert np.array_equal(d, om.desc) and np.array_equal(s, exp), (rep, j)
    g.close()


def test_graph_duplicate_is_reported_per_map(F):
    b = W.batched_workload(6, 100, 2000, 100, 0.75, seed=19)
    keys = b.keys.copy()
    keys[b.seg_offs[4] + 3] = keys[b.seg_offs[4]]
    g = F.fks_build_graph_create(F.FKS_KEY_U64, dev(keys), None, None, b.seg_offs, dev(b.vals))
    st = F.fks_build_graph_run(g, b.seeds, raise_on_error=False)
    assert st.tolist() == [0, 0, 0, 0, F.FKS_ERR_DUPLICATE_KEY, 0]
    S = g.mapset()
    assert S.get(4) is None
    check_u64_maps(F, S, keys, b.vals, b.seg_offs, b.seeds, [0, 5])
    g.close()


def test_graph_rejects_dedup(F):
    b = W.batched_workload(2, 16, 64, 10, 0.5, seed=3)
    with pytest.raises(F.FksError) as e:
        F.fks_build_graph_create(F.FKS_KEY_U64, dev(b.keys), None, None, b.seg_offs, dev(b.vals),
                                 opts=F.make_opts(dedup=1))
    assert e.value.status == F.FKS_ERR_INVALID_ARG
