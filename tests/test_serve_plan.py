"""Host logic of the serving workload (no GPU): the LRU model that makes every
lookup target a resident map under the budget."""
import collections

import numpy as np

from paper_2508_11443_b300 import workloads as W


def test_plan_lookups_target_resident_maps_within_budget():
    s = W.string_workload(1 << 12, 8, 0.0, seed=2)
    budget = 4 << 20
    P = W.serving_plan(3000, 5, budget, s.offs, prefill=16, u64_n=(2**10, 2**14), str_n=(2**10, 2**11),
                       nq_range=(1, 2**10), u64_pool=2**16)
    assert (P.kind[:16] == 0).all()
    resident = collections.OrderedDict()
    used = 0
    for r in range(P.kind.size):
        if P.kind[r] == 0:
            o, n = int(P.off[r]), int(P.n[r])
            need = (W.STR_MAP_BYTES_PER_KEY * n + int(s.offs[o + n] - s.offs[o])) if P.key_kind[r] \
                else W.U64_MAP_BYTES_PER_KEY * n
            while used + need > budget:
                _, b = resident.popitem(last=False)
                used -= b
            resident[int(P.map_id[r])] = need
            used += need
            assert used <= budget
        else:
            assert int(P.map_id[r]) in resident
            resident.move_to_end(int(P.map_id[r]))
            assert 0 <= P.nhit[r] <= P.nq[r]
    frac = P.nhit[P.kind == 1].sum() / P.nq[P.kind == 1].sum()
    assert abs(frac - 0.8) < 0.02
    assert abs((P.kind[16:] == 1).mean() - 0.9) < 0.03
    # map ids are unique per build
    ids = P.map_id[P.kind == 0]
    assert np.array_equal(ids, np.arange(ids.size))


def test_poisson_arrivals_rate():
    a = W.poisson_arrivals_us(20000, 1e5, 1)
    assert np.all(np.diff(a) > 0)
    assert abs(a[-1] / 20000 - 10.0) < 0.3  # mean gap 10 us
