"""The several-GPU path of bench.py (replicas, weak scaling) on CPU: two gloo
ranks launched like torchrun (RANK / WORLD_SIZE / MASTER_* in the
environment) agree on the slowest rank's time, use distinct key streams,
and count the work of both ranks."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    from paper_2508_11443_b300 import workloads as W
    w_, r_, l_ = bench.dist_setup()
    dist.init_process_group("gloo", rank=r_, world_size=w_)
    my_ms = 10.0 * (rank + 1) + 0.25
    ms = bench.max_over_ranks(my_ms, w_, "cpu")
    keys = W.u64_workload(64, 8, 0.5, bench.rank_seed(r_)).keys
    dist.barrier()
    res = {"rank": r_, "world": w_, "local": l_, "ms": ms, "seed": bench.rank_seed(r_),
           "first_key": int(keys[0]), "value": bench.job_throughput(1000, w_, ms)}
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    assert [r["rank"] for r in res] == [0, 1] and all(r["world"] == 2 for r in res)
    assert all(r["ms"] == pytest.approx(20.25) for r in res)  # the slowest rank's time, on every rank
    assert res[0]["seed"] != res[1]["seed"] and res[0]["first_key"] != res[1]["first_key"]
    assert res[0]["value"] == pytest.approx(2 * 1000 / (20.25 / 1e3))


def test_single_process_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(100, 1, 1.0) == pytest.approx(1e5)
