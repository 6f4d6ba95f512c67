"""Benchmark of the FKS hot path on one B300 (or N replicas under torchrun).

A step is one pass of the whole path over one batch of synthetic input:
build of a map over 2^26 distinct uint64 keys (int64 values) followed by a
lookup batch of 2^26 queries at a 90 % hit rate against it (uniform hits,
exact non-members for the misses), then the map is released.  Inputs are
resident in HBM before the timed region (512 MiB per array, far larger than
the 126 MB L2, so no flush is needed between steps).

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FKS build keys/s & lookups/s (% HBM roofline); served p50/p99 vs per-call"
N_KEYS = 1 << 26
N_QUERIES = 1 << 26
HIT = 0.9
SEED = 2
WORKLOAD = "u64 build 2^26 keys + lookup 2^26 queries (90% hits)"

# algorithmic bytes (32-byte sector model) -- see the design notes
SECTOR = 32


def lookup_bytes_per_query(hit_frac: float, nonempty_frac: float) -> float:
    """needle 8 + descriptor sector + slot sector (hits, and misses that land
    in a non-empty bucket) + value 8 + found flag 1."""
    return 8 + SECTOR + SECTOR * (hit_frac + (1 - hit_frac) * nonempty_frac) + 8 + 1


def part_build_bytes_per_key(S_over_n: float) -> float:
    """staged key+value read 16 + descriptor write 8 + slot writes 16 * S/n."""
    return 16 + 8 + 16 * S_over_n


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def load_traffic():
    """DRAM bytes per launch from the committed ncu summary, keyed by kernel,
    with the kernel source digest they were taken at."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    out = {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        m = re.match(r"\|\s*(k_\w+)\s*\|\s*([0-9.eE+]+)\s*\|\s*([0-9a-f]{12})\s*\|", line)
        if m:
            out[m.group(1)] = (float(m.group(2)), m.group(3))
    return out


def kernel_traffic(kernel: str, units: int):
    """DRAM bytes of one launch over `units` keys or queries, scaled from the
    committed 2^26 figure; None once the kernel's sources have changed since
    the counters were taken."""
    t = load_traffic()
    if kernel in t and t[kernel][1] == kernel_digest(kernel):
        return t[kernel][0] * units / float(1 << 26)
    return None


# source files each kernel is compiled from (digest ties ncu counters to code)
KERNEL_SOURCES = {
    "k_lookup_u64": ["fks_device.cuh", "fks_internal.cuh", "fks_strings.cuh", "fks_lookup.cu"],
    "k_part_build": ["fks_device.cuh", "fks_internal.cuh", "fks_strings.cuh", "fks_build.cu"],
    "k_partition_scatter": ["fks_device.cuh", "fks_internal.cuh", "fks_strings.cuh", "fks_build.cu"],
    "k_partition_count": ["fks_device.cuh", "fks_internal.cuh", "fks_strings.cuh", "fks_build.cu"],
    "k_scatterA": ["fks_device.cuh", "fks_internal.cuh", "fks_split.cu"],
    "k_scatterB": ["fks_device.cuh", "fks_internal.cuh", "fks_split.cu"],
    "k_lookup_inline": ["fks_device.cuh", "fks_internal.cuh", "fks_strings.cuh", "fks_lookup.cu"],
}


def kernel_digest(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2508_11443_b300", "csrc")
    for f in sorted(KERNEL_SOURCES[kernel]):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:12]


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled through NVML every
    few milliseconds from a background thread (read-only queries).  mark()
    brackets the timed region; summary() keeps the samples inside it."""

    REASONS = (("hw_slowdown", "nvmlClocksEventReasonHwSlowdown"),
               ("hw_thermal_slowdown", "nvmlClocksEventReasonHwThermalSlowdown"),
               ("sw_thermal_slowdown", "nvmlClocksEventReasonSwThermalSlowdown"),
               ("sw_power_cap", "nvmlClocksEventReasonSwPowerCap"),
               ("hw_power_brake", "nvmlClocksEventReasonHwPowerBrakeSlowdown"))

    def __init__(self, index: int, period_s: float = 0.002):
        self.index, self.period = index, period_s
        self.samples = []  # (t, sm_mhz, reasons bitmask)
        self.window = None
        self.max_mhz = None
        self.err = None

    def __enter__(self):
        try:
            import pynvml
            pynvml.nvmlInit()
            self.nv = pynvml
            self.h = pynvml.nvmlDeviceGetHandleByIndex(self.index)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._run, daemon=True)
            self.thread.start()
        except Exception as e:  # no NVML binding: nvidia-smi queries instead
            self.err = repr(e)
            self._start_smi()
        return self

    # bit values of the NVML clock-event reasons, for the nvidia-smi fallback
    SMI_BITS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
                "sw_power_cap": 0x4, "hw_power_brake": 0x80}

    def _start_smi(self):
        import subprocess
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap,clocks_event_reasons.hw_power_brake_slowdown")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "10"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read_smi, daemon=True)
            self.thread.start()
            time.sleep(0.5)  # let nvidia-smi start before the timed region
        except Exception as e:
            self.err = repr(e)
            self.proc = None

    def _read_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap", "hw_power_brake"]
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) != 7:
                continue
            try:
                sm = float(parts[0])
                self.max_mhz = float(parts[1])
            except ValueError:
                continue
            mask = 0
            for name, val in zip(names, parts[2:]):
                if val == "Active":
                    mask |= self.SMI_BITS[name]
            self.samples.append((time.perf_counter(), sm, mask))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *a):
        if hasattr(self, "stop"):
            self.stop.set()
            self.thread.join(timeout=2)
        if getattr(self, "proc", None) is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples: " + str(self.err)]}
        t0, t1 = self.window or (self.samples[0][0], self.samples[-1][0])
        inside = [s for s in self.samples if t0 <= s[0] <= t1] or \
            sorted(self.samples, key=lambda s: min(abs(s[0] - t0), abs(s[0] - t1)))[:3]
        mask = 0
        for s in inside:
            mask |= int(s[2])
        reasons = [name for name, _ in self.REASONS if mask & self.SMI_BITS[name]]
        return {"sm_mhz": statistics.median(s[1] for s in inside), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(inside)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# Several GPUs run replicas (weak scaling): every rank builds and queries a
# map of its own from its own key stream, with no collective in the data
# path; the job's time is the slowest rank's and its throughput counts the
# work of all ranks.
def rank_seed(rank: int) -> int:
    return SEED + rank


def max_over_ranks(ms: float, world: int, device) -> float:
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_per_step: float) -> float:
    return units_per_rank * world / (ms_per_step / 1e3)


def cpu_sample_run(n: int, nq: int, seed: int):
    """Oracle build + lookup over a sample of the workload; returns seconds."""
    import oracle as O
    from paper_2508_11443_b300 import workloads as W
    w = W.u64_workload(n, nq, HIT, seed)
    t0 = time.perf_counter()
    m = O.build_u64(w.keys, w.vals, seed=seed)
    out, found = O.lookup_u64(m, w.queries)
    dt = time.perf_counter() - t0
    assert m.status == O.OK and np.array_equal(found, w.expect_found)
    return dt


def run_reference(args, world, rank):
    if rank != 0:
        return
    n = min(args.cpu_sample, 1 << 22)
    times = []
    for i in range(args.warmup + args.steps):
        dt = cpu_sample_run(n, n, SEED + 1000 + i)
        if i >= args.warmup:
            times.append(dt)
    per_step = statistics.mean(times)
    value = 2 * n / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "keys+lookups/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_keys": N_KEYS, "n_queries": N_QUERIES, "hit_rate": HIT,
                   "sample": f"each step: oracle build of {n} keys + lookup of {n} queries"},
        "cpu_baseline": {"value": value, "unit": "keys+lookups/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n} keys built + {n} queries per step, single thread"},
        "e2e": {"value": value, "unit": "keys+lookups/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _timed(torch, stream, fn, reps=3, warm=1):
    ts = []
    for i in range(warm + reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        if i >= warm:
            ts.append(a.elapsed_time(b))
        del r
    return statistics.median(ts)


def run_strings(F, W, torch, hbm, shift=0):
    """String keys: 2^22 distinct strings (lengths uniform in [4, 64], a-z) with
    int32 values; 2^24 needles, 50 % members."""
    w = W.string_workload(1 << (22 - shift), 1 << (24 - shift), 0.5, seed=3)
    ctx, offs = torch.from_numpy(w.ctx).cuda(), torch.from_numpy(w.offs).cuda()
    vals = torch.from_numpy(w.vals.astype(np.int32)).cuda()
    qctx, qoffs = torch.from_numpy(w.qctx).cuda(), torch.from_numpy(w.qoffs).cuda()
    nq = w.qoffs.size - 1
    out = torch.empty(nq, dtype=torch.int32, device="cuda")
    found = torch.empty(nq, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    bms = _timed(torch, stream, lambda: F.fks_build_bytes(ctx, offs, vals, 3))
    m = F.fks_build_bytes(ctx, offs, vals, 3)
    lms = _timed(torch, stream, lambda: F.fks_lookup_bytes(m, qctx, qoffs, out, found, -1))
    ok = np.array_equal(found.cpu().numpy(), w.expect_found)
    info = F.fks_map_info(m)
    L = float(np.diff(w.offs).mean())
    Lq = float(np.diff(w.qoffs).mean())
    ne = info.nonempty_buckets / info.n
    # needle: offsets 8 + bytes + descriptor sector + slot sector (hits, misses in
    # non-empty buckets) + on a hit the map's context span (1 + (L-1)/32 sectors)
    # + value 4 + found 1
    lq = 8 + Lq + 32 + 32 * (0.5 + 0.5 * ne) + 0.5 * 32 * (1 + (L - 1) / 32) + 4 + 1
    n = w.offs.size - 1
    return {"workload": "2^22 strings (4..64 bytes, a-z), int32 values; 2^24 needles, 50% members",
            "build_ms": bms, "build_keys_per_s": n / (bms / 1e3), "lookup_ms": lms,
            "lookups_per_s": nq / (lms / 1e3), "lookup_bytes_model": f"{lq:.1f} B/needle",
            "lookup_GBps": lq * nq / (lms / 1e3) / 1e9, "lookup_frac": lq * nq / (lms / 1e3) / 1e9 / hbm,
            "results_match_truth": bool(ok), "S_over_n": info.slots / info.n}


def run_batched(F, W, torch, hbm, shift=0):
    """Batched maps: 1024 maps of log-uniform size in [16, 2^20] built by one
    batched call; 2^24 (map_id, key) lookups at 75 % hits."""
    b = W.batched_workload(1024 >> shift, 16, 1 << (20 - shift), 1 << (24 - shift), 0.75, seed=4)
    keys = torch.from_numpy(b.keys.view(np.int64)).cuda()
    vals = torch.from_numpy(b.vals).cuda()
    ids = torch.from_numpy(b.q_map.astype(np.int32)).cuda()
    q = torch.from_numpy(b.q_keys.view(np.int64)).cuda()
    out = torch.empty(q.numel(), dtype=torch.int64, device="cuda")
    found = torch.empty(q.numel(), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    total = int(b.seg_offs[-1])
    bms = _timed(torch, stream, lambda: F.fks_build_batched(F.FKS_KEY_U64, keys, None, None, b.seg_offs, b.seeds,
                                                              vals))
    S = F.fks_build_batched(F.FKS_KEY_U64, keys, None, None, b.seg_offs, b.seeds, vals)
    lms = _timed(torch, stream, lambda: F.fks_lookup_batched(S, ids, q=q, out_vals=out, out_found=found))
    ok = np.array_equal(found.cpu().numpy(), b.expect_found)
    lq = 4 + 8 + 32 + 32 * (0.75 + 0.25 * 0.632) + 8 + 1
    return {"workload": "%d maps, n log-uniform in [16, 2^%d] (sum %d keys); 2^%d lookups, 75%% hits" % (
                1024 >> shift, 20 - shift, total, 24 - shift),
            "build_ms": bms, "build_keys_per_s": total / (bms / 1e3), "lookup_ms": lms,
            "lookups_per_s": q.numel() / (lms / 1e3), "lookup_bytes_model": f"{lq:.1f} B/query",
            "lookup_GBps": lq * q.numel() / (lms / 1e3) / 1e9,
            "lookup_frac": lq * q.numel() / (lms / 1e3) / 1e9 / hbm, "results_match_truth": bool(ok)}


def run_graph_builds(F, W, torch, shift=0):
    """Batched builds as one recorded CUDA graph (fks_build_graph_run) against
    the same batched build launched pass by pass (fks_build_batched) and, for
    small maps, against one fks_build_u64 call per map: the 1024 batched maps
    of log-uniform size in [16, 2^20], and 2048 small maps of log-uniform size
    in [16, 4096], where launch and synchronisation costs dominate."""
    stream = torch.cuda.current_stream()
    res = {}
    for name, m, lo, hi, per_call in (("batched_1024_maps", 1024 >> shift, 16, 1 << (20 - shift), False),
                                      ("small_2048_maps", 2048 >> shift, 16, 4096, True)):
        b = W.batched_workload(m, lo, hi, 16, 0.75, seed=4)
        keys = torch.from_numpy(b.keys.view(np.int64)).cuda()
        vals = torch.from_numpy(b.vals).cuda()
        total = int(b.seg_offs[-1])
        bms = _timed(torch, stream, lambda: F.fks_build_batched(F.FKS_KEY_U64, keys, None, None, b.seg_offs,
                                                                  b.seeds, vals), reps=5)
        g = F.fks_build_graph_create(F.FKS_KEY_U64, keys, None, None, b.seg_offs, vals)
        gms = _timed(torch, stream, lambda: F.fks_build_graph_run(g, b.seeds), reps=5)
        st = F.fks_build_graph_run(g, b.seeds)
        S = g.mapset()
        ok = bool((st == 0).all())
        for j in (0, m // 2, m - 1):  # the graph's tables equal a per-call build's
            k0, k1 = int(b.seg_offs[j]), int(b.seg_offs[j + 1])
            pm = F.fks_build_u64(keys[k0:k1], vals[k0:k1], int(b.seeds[j]))
            d1, s1, _ = F.fks_map_export(S.get(j))
            d2, s2, _ = F.fks_map_export(pm)
            ok = ok and np.array_equal(d1, d2) and np.array_equal(s1, s2)
        r = {"maps": m, "keys": total, "batched_ms": bms, "graph_ms": gms,
             "graph_kernels": g.kernels(), "graph_speedup": bms / gms,
             "graph_keys_per_s": total / (gms / 1e3), "tables_match_per_call": ok}
        if per_call:
            segs = [(int(b.seg_offs[j]), int(b.seg_offs[j + 1]), int(b.seeds[j])) for j in range(m)]

            def loop():
                for k0, k1, sd in segs:
                    F.fks_build_u64(keys[k0:k1], vals[k0:k1], sd)
            pms = _timed(torch, stream, loop, reps=3)
            r["per_call_ms"] = pms
            r["graph_speedup_over_per_call"] = pms / gms
        del S
        g.close()
        res[name] = r
        torch.cuda.empty_cache()
    return res


# The paper's Table 1 (an A100, Futhark; ms for 10^7 keys): construction,
# lookup, membership.  Context for the row below, not a target.
PAPER_TABLE1_A100_MS = {
    "fks_u64": (18.3, 3.3, 1.6), "binary_search_u64": (40.9, 6.2, 5.8), "eytzinger_u64": (42.3, 4.3, 2.4),
    "cucollections_u64": (2.7, 1.1, 0.9), "fks_strings": (33.2, 4.3, 2.8)}


def run_paper_table1(F, W, torch):
    """The paper's own evaluation setup: n = 10^7 distinct keys with int32
    values; lookup (value + presence) and membership (presence only) of every
    inserted key, so 100 % hits; uint64 keys, and strings of 5-25 lowercase
    letters.  The search-based maps on the same uint64 keys."""
    stream = torch.cuda.current_stream()
    n = 10_000_000
    keys_h = W.key_stream(71, n)
    keys = torch.from_numpy(keys_h.view(np.int64)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    found = torch.empty(n, dtype=torch.uint8, device="cuda")
    res = {"workload": "10^7 distinct keys, int32 values, every key looked up (100 % hits)",
           "paper_a100_ms": {k: {"build": v[0], "lookup": v[1], "membership": v[2]}
                             for k, v in PAPER_TABLE1_A100_MS.items()}}

    def row(build, lookup, member):
        bms = _timed(torch, stream, build)
        mp = build()
        lms = _timed(torch, stream, lambda: lookup(mp))
        ok = bool(found.all().item()) and bool(torch.equal(out, vals))
        mms = _timed(torch, stream, lambda: member(mp))
        ok = ok and bool(found.all().item())
        del mp
        return {"build_ms": bms, "lookup_ms": lms, "membership_ms": mms, "all_found": ok}

    res["fks_u64"] = row(lambda: F.fks_build_u64(keys, vals, 7),
                         lambda mp: F.fks_lookup_u64(mp, keys, out, found, -1),
                         lambda mp: F.fks_lookup_u64(mp, keys, None, found, -1))
    res["binary_search_u64"] = row(lambda: F.fks_sortmap_build(keys, vals),
                                   lambda mp: F.fks_sortmap_lookup(mp, keys, out, found, -1),
                                   lambda mp: F.fks_sortmap_lookup(mp, keys, None, found, -1))
    res["eytzinger_u64"] = row(lambda: F.fks_eytzmap_build(keys, vals),
                               lambda mp: F.fks_sortmap_lookup(mp, keys, out, found, -1),
                               lambda mp: F.fks_sortmap_lookup(mp, keys, None, found, -1))
    sw = W.string_workload(n, 1, 1.0, seed=72, lo=5, hi=25)
    ctx, offs = torch.from_numpy(sw.ctx).cuda(), torch.from_numpy(sw.offs).cuda()
    res["fks_strings"] = row(lambda: F.fks_build_bytes(ctx, offs, vals, 8),
                             lambda mp: F.fks_lookup_bytes(mp, ctx, offs, out, found, -1),
                             lambda mp: F.fks_lookup_bytes(mp, ctx, offs, None, found, -1))
    for k, r in res.items():
        if k in PAPER_TABLE1_A100_MS:
            pb, pl, pm = PAPER_TABLE1_A100_MS[k]
            r["vs_paper_a100"] = {"build": pb / r["build_ms"], "lookup": pl / r["lookup_ms"],
                                  "membership": pm / r["membership_ms"]}
    del keys, vals, out, found, ctx, offs
    torch.cuda.empty_cache()
    return res


def run_bucket_variants(F, torch, hbm, keys, vals, queries, out, found, w, n, nq, tune=True):
    """The level-one bucket-count variant on the headline workload: nb =
    ceil(n / lambda) buckets for lambda in 1, 2, 4, 8, 16 (1 is the paper's
    construction).  Fewer buckets keep the descriptor array (8 nb bytes) in
    L2, so lookups approach one DRAM access per query; the slot array grows
    to about (1 + lambda) n slots.  Each lambda runs at the launch shapes the
    autotuner measured for it on this size (tune=False: the current table)."""
    stream = torch.cuda.current_stream()
    res = {}
    for lam in (1, 2, 4, 8, 16):
        if tune and lam > 1:
            F.fks_autotune(F.FKS_KEY_U64, lam, n=n, nq=nq, seed=SEED + lam)
        o = F.make_opts(keys_per_bucket=lam)
        bms = _timed(torch, stream, lambda: F.fks_build_u64(keys, vals, SEED, o))
        m = F.fks_build_u64(keys, vals, SEED, o)
        lms = _timed(torch, stream, lambda: F.fks_lookup_u64(m, queries, out, found, -1))
        ok = np.array_equal(found.cpu().numpy(), w.expect_found) and \
            np.array_equal(out.cpu().numpy(), np.where(w.expect_found == 1, w.expect_vals, -1))
        info = F.fks_map_info(m)
        ne = info.nonempty_buckets / info.buckets
        lq = lookup_bytes_per_query(HIT, ne)
        res[str(lam)] = {
            "buckets": int(info.buckets), "descriptor_MB": info.buckets * 8 / 1e6,
            "S_over_n": info.slots / n, "map_bytes_per_key": info.bytes / n,
            "build_ms": bms, "lookup_ms": lms, "step_ms": bms + lms,
            "build_keys_per_s": n / (bms / 1e3), "lookups_per_s": nq / (lms / 1e3),
            "keys_plus_lookups_per_s": (n + nq) / ((bms + lms) / 1e3),
            "lookup_bytes_model": f"{lq:.2f} B/query", "lookup_GBps": lq * nq / (lms / 1e3) / 1e9,
            "lookup_frac": lq * nq / (lms / 1e3) / 1e9 / hbm, "results_match_truth": bool(ok),
            "shape": {k: v for k, v in F.fks_tuning_get(F.FKS_KEY_U64, lam).as_dict().items()
                      if k in ("thread_search_max", "split_min_keys_log2", "lookup_queries_per_thread",
                               "lookup_block", "lookup_blocks_per_sm", "tuned")}}
        del m
        torch.cuda.empty_cache()
    return res


def run_inline_singletons(F, torch, hbm, keys, vals, queries, out, found, w, n, nq):
    """The inline-singleton records (build option inline_singletons) on the
    headline workload: the paper's tables plus a 16-byte record per bucket, so
    a needle whose bucket holds no key or one key is answered by one random
    access.  Byte model (32-byte sectors, a Poisson(1) bucket-size law): needle
    8 + record sector + a slot sector for hits in buckets of two or more keys
    (1 - 1/e of the hits) and misses that land in such a bucket (1 - 2/e) +
    value 8 + flag 1."""
    stream = torch.cuda.current_stream()
    o = F.make_opts(inline_singletons=1)
    bms = _timed(torch, stream, lambda: F.fks_build_u64(keys, vals, SEED, o))
    m = F.fks_build_u64(keys, vals, SEED, o)
    lms = _timed(torch, stream, lambda: F.fks_lookup_u64(m, queries, out, found, -1))
    ok = np.array_equal(found.cpu().numpy(), w.expect_found) and \
        np.array_equal(out.cpu().numpy(), np.where(w.expect_found == 1, w.expect_vals, -1))
    info = F.fks_map_info(m)
    e1 = float(np.exp(-1.0))
    lq = 8 + SECTOR + SECTOR * (HIT * (1 - e1) + (1 - HIT) * (1 - 2 * e1)) + 8 + 1
    del m
    torch.cuda.empty_cache()
    return {"workload": "the headline workload, map built with inline-singleton records",
            "build_ms": bms, "lookup_ms": lms, "step_ms": bms + lms,
            "map_bytes_per_key": info.bytes / n, "build_keys_per_s": n / (bms / 1e3),
            "lookups_per_s": nq / (lms / 1e3), "keys_plus_lookups_per_s": (n + nq) / ((bms + lms) / 1e3),
            "lookup_bytes_model": f"{lq:.2f} B/query", "lookup_GBps": lq * nq / (lms / 1e3) / 1e9,
            "lookup_frac": lq * nq / (lms / 1e3) / 1e9 / hbm, "results_match_truth": bool(ok),
            "lookup_traffic": kernel_traffic("k_lookup_inline", nq)}


def run_from_array(F, W, torch, hbm, shift=0):
    """from_array (opts.dedup = 1): 2^26 pairs whose keys are drawn with
    replacement from 2^25 distinct keys (about 2.9e7 distinct); the first
    occurrence wins.  Timed: the deduplicating pre-pass + the build."""
    u, universe = 1 << (26 - shift), 1 << (25 - shift)
    rng = np.random.default_rng(17)
    base = W.key_stream(17, universe)
    keys_h = base[rng.integers(0, universe, u)]
    keys = torch.from_numpy(keys_h.view(np.int64)).cuda()
    vals = torch.from_numpy(np.arange(u, dtype=np.int64)).cuda()
    stream = torch.cuda.current_stream()
    o = F.make_opts(dedup=1)
    ms = _timed(torch, stream, lambda: F.fks_build_u64(keys, vals, 5, o))
    m = F.fks_build_u64(keys, vals, 5, o)
    info = F.fks_map_info(m)
    # first occurrence check on a sample: the map returns the index of the first occurrence
    first = {}
    for e, k in enumerate(keys_h[: 1 << 16].tolist()):
        first.setdefault(k, e)
    q = np.fromiter(first.keys(), np.uint64)
    out = torch.empty(q.size, dtype=torch.int64, device="cuda")
    F.fks_lookup_u64(m, torch.from_numpy(q.view(np.int64)).cuda(), out, None, -1)
    torch.cuda.synchronize()
    ok = np.array_equal(out.cpu().numpy(), np.fromiter(first.values(), np.int64))
    # pre-pass bytes: insert (key 8 + table sector 32 + value-free) + keep (key 8 + sector 32 + flag 4)
    # + scan (8) + pack (pos 8 + key 8 + value 8 + writes 16)
    dd = (8 + 32) + (8 + 32 + 4) + 8 + (8 + 16 + 16)
    del m
    torch.cuda.empty_cache()
    return {"workload": "2^%d u64 pairs, keys drawn from 2^%d distinct, first occurrence wins" % (26 - shift,
                                                                                               25 - shift),
            "distinct_keys": int(info.n), "dedup_plus_build_ms": ms,
            "input_pairs_per_s": u / (ms / 1e3), "prepass_bytes_model": f"{dd} B/pair",
            "first_occurrence_sample_ok": bool(ok)}


def run_serving(args, F, W, torch):
    """Serving: a Poisson stream of build and lookup requests (90 % lookups of
    log-uniform size in [1, 2^16], 80 % hits; 10 % builds, half uint64 maps of
    log-uniform size in [2^10, 2^22], half string maps in [2^10, 2^20]) over
    maps resident under a 40 GB budget with LRU eviction, after 64 prefill
    builds.  The per-call server's saturation throughput mu is measured with
    every request arriving at once; both servers then replay the same stream
    at lambda = rho * mu.  Latency: submission to completion seen on the host."""
    strings = W.string_workload(1 << 20, 1 << 20, 0.0, seed=55)
    plan = W.serving_plan(args.serve_requests, 77, 40 << 30, strings.offs)
    data = W.ServeData(plan, seed=78, strings=strings)
    exp_found = None
    pre = plan.prefill

    def once(mode, arrival):
        srv = F.fks_server_create(memory_budget=plan.budget, max_maps=int(plan.map_id.max()) + 1, mode=mode)
        # prefill builds (outside the clock), then the timed stream
        F.fks_server_replay(srv, data.reqs, np.zeros(pre))
        F.fks_server_drain(srv)
        import ctypes
        stream_reqs = (F.fks_request * (plan.kind.size - pre)).from_address(
            ctypes.addressof(data.reqs) + pre * ctypes.sizeof(F.fks_request))
        tickets = F.fks_server_replay(srv, stream_reqs, arrival)
        F.fks_server_drain(srv)
        res = [F.fks_server_wait(srv, int(t)) for t in tickets]
        st = F.fks_server_stats(srv)
        srv.close()
        lat = np.array([l for _, l in res])
        ok = np.array([s == F.FKS_OK for s, _ in res])
        kinds = plan.kind[pre:]
        span = (max(arrival[-1], 0) + 0.0) / 1e6
        t_last = max(arrival[i] + lat[i] for i in range(lat.size)) / 1e6
        return {"p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                "lookup_p50_us": float(np.percentile(lat[kinds == 1], 50)),
                "lookup_p99_us": float(np.percentile(lat[kinds == 1], 99)),
                "build_p50_us": float(np.percentile(lat[kinds == 0], 50)),
                "build_p99_us": float(np.percentile(lat[kinds == 0], 99)),
                "throughput_req_per_s": lat.size / t_last, "queries_per_s": float(plan.nq[pre:].sum()) / t_last,
                "failed": int((~ok).sum()), "lookup_batches": int(st.batches), "evictions": int(st.evictions),
                "peak_resident_gb": st.peak_resident_bytes / 1e9}

    m = plan.kind.size - pre
    sat = once(F.FKS_SERVE_PER_CALL, np.zeros(m))
    mu = sat["throughput_req_per_s"]
    # saturation of the batched server on the same stream (every request at once)
    sat_b = once(F.FKS_SERVE_BATCHED, np.zeros(m))
    out = {"requests": m, "prefill_builds": pre, "budget_gb": 40, "mu_per_call_req_per_s": mu,
           "mu_batched_req_per_s": sat_b["throughput_req_per_s"],
           "saturation_throughput_ratio_batched_over_per_call": sat_b["throughput_req_per_s"] / mu,
           "rho": args.serve_rho, "rate_req_per_s": args.serve_rho * mu}
    arrival = W.poisson_arrivals_us(m, args.serve_rho * mu, 5)
    out["per_call"] = once(F.FKS_SERVE_PER_CALL, arrival)
    out["batched"] = once(F.FKS_SERVE_BATCHED, arrival)
    over = W.poisson_arrivals_us(m, 1.2 * mu, 6)
    out["over_saturation_rho_1_2"] = {"per_call": once(F.FKS_SERVE_PER_CALL, over),
                                      "batched": once(F.FKS_SERVE_BATCHED, over)}
    # the batched run's results against the stream's truth
    f = data.found.cpu().numpy()
    looks = np.nonzero(plan.kind == 1)[0]
    want = np.concatenate([data.u_hit.cpu().numpy().astype(np.uint8) if data.u_index else np.zeros(0, np.uint8),
                           data.s_hit.cpu().numpy().astype(np.uint8) if data.s_index else np.zeros(0, np.uint8)])
    got = np.concatenate([np.concatenate([f[data.out_start[r]:data.out_start[r] + plan.nq[r]]
                                          for r in looks if plan.key_kind[r] == k] or [np.zeros(0, np.uint8)])
                          for k in (0, 1)])
    out["batched_results_match_truth"] = bool(np.array_equal(got, want))
    out["p99_ratio_per_call_over_batched"] = out["per_call"]["p99_us"] / max(out["batched"]["p99_us"], 1e-9)
    out["throughput_ratio_batched_over_per_call"] = (out["batched"]["throughput_req_per_s"] /
                                                    out["per_call"]["throughput_req_per_s"])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fks", choices=["fks", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=1 << 24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-search-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--serve-rho", type=float, default=0.8)
    ap.add_argument("--n", type=int, default=N_KEYS)
    ap.add_argument("--no-autotune", action="store_true")
    # install these launch-shape fields (uint64 keys, one bucket per key)
    # instead of running the autotuner, e.g. lookup_block=512,lookup_blocks_per_sm=1024
    ap.add_argument("--tuning", default="")
    # the string, batched, graph and from_array rows at 2^-shift of their
    # sizes (small cases for profiler captures); 0 = the configured sizes
    ap.add_argument("--extras-shift", type=int, default=0)
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import torch.distributed as dist
    from paper_2508_11443_b300 import build as B
    from paper_2508_11443_b300 import fks as F
    from paper_2508_11443_b300 import workloads as W

    assert args.warmup >= 3, "at least 3 warm-up steps"
    B.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.n
    nq = n
    w = W.u64_workload(n, nq, HIT, rank_seed(rank))
    keys = torch.from_numpy(w.keys.view(np.int64)).cuda()
    vals = torch.from_numpy(w.vals).cuda()
    queries = torch.from_numpy(w.queries.view(np.int64)).cuda()
    out = torch.empty(nq, dtype=torch.int64, device="cuda")
    found = torch.empty(nq, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    # launch shapes of the build and the lookup, measured on this workload's
    # size before anything is timed (the timed step then runs at them)
    tune = None
    if args.tuning:
        entry = F.fks_tuning_get(F.FKS_KEY_U64, 1)
        for kv in args.tuning.split(","):
            k, v = kv.split("=")
            setattr(entry, k.strip(), int(v))
        F.fks_tuning_set(entry)
        tune = {"installed": entry.as_dict()}
    elif not args.no_autotune:
        t0 = time.perf_counter()
        entry, trials = F.fks_autotune(F.FKS_KEY_U64, 1, n=n, nq=nq, seed=rank_seed(rank) + 1)
        tune = {"seconds": time.perf_counter() - t0, "entry": entry.as_dict(),
                "trials": [[p, v, round(ms, 4)] for p, v, ms in trials]}
    F.fks_profile_enable(True)

    build_ms, part_ms, lookup_ms, step_ms, nonempty, S = [], [], [], [], [], []

    def step(timed):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        m = F.fks_build_u64(keys, vals, rank_seed(rank))
        e1.record(stream)
        F.fks_lookup_u64(m, queries, out, found, -1)
        e2.record(stream)
        if timed:
            prof = F.fks_last_build_profile()
            info = F.fks_map_info(m)
            torch.cuda.synchronize()
            build_ms.append(e0.elapsed_time(e1))
            lookup_ms.append(e1.elapsed_time(e2))
            step_ms.append(e0.elapsed_time(e2))
            part_ms.append((prof.count_ms, prof.scan_ms, prof.scatter_ms, prof.part_build_ms,
                            prof.group_ms, prof.grouping_levels))
            nonempty.append(info.nonempty_buckets / info.n)
            S.append(info.slots / info.n)
        del m

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    # correctness of the last warm-up lookup
    f = found.cpu().numpy()
    o = out.cpu().numpy()
    assert np.array_equal(f, w.expect_found), "lookup found flags differ from the workload's truth"
    assert np.array_equal(o, np.where(w.expect_found == 1, w.expect_vals, -1)), "lookup values differ"

    launches0 = F.fks_kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.05)
        h0 = time.perf_counter()
        t_start.record(stream)
        for _ in range(args.steps):
            step(True)
        t_end.record(stream)
        torch.cuda.synchronize()
        clk.mark(h0, time.perf_counter())
        if world > 1:
            dist.barrier()
    launches = F.fks_kernel_launches() - launches0
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), world, "cuda")
    ms_per_step = total_ms / args.steps
    units = (n + nq) * world
    value = job_throughput(n + nq, world, ms_per_step)

    # ---- end to end through the C ABI from pinned host memory
    h_keys = torch.from_numpy(w.keys.view(np.int64)).pin_memory()
    h_vals = torch.from_numpy(w.vals).pin_memory()
    h_q = torch.from_numpy(w.queries.view(np.int64)).pin_memory()
    h_out = torch.empty(nq, dtype=torch.int64).pin_memory()
    h_found = torch.empty(nq, dtype=torch.uint8).pin_memory()

    def e2e_step():
        # the host-buffer entry points: upload + build, then needles streamed
        # through the device in chunks (upload, lookup and download overlap)
        m = F.fks_build_u64_host(h_keys, h_vals, rank_seed(rank))
        F.fks_lookup_u64_host(m, h_q, h_out, h_found, -1)
        del m

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(3, args.steps // 2)
    a.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(a.elapsed_time(b) / e2e_steps, world, "cuda")
    assert np.array_equal(h_found.numpy(), w.expect_found)
    # where the end-to-end time goes: the two host-buffer calls, and the host
    # link's own pinned copy rates (outside the timed region)
    c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    c0.record(stream)
    m_e = F.fks_build_u64_host(h_keys, h_vals, rank_seed(rank))
    c1.record(stream)
    F.fks_lookup_u64_host(m_e, h_q, h_out, h_found, -1)
    c2.record(stream)
    torch.cuda.synchronize()
    del m_e
    d_tmp = torch.empty_like(keys)
    h2d_ms = _timed(torch, stream, lambda: d_tmp.copy_(h_keys, non_blocking=True), reps=3)
    d2h_ms = _timed(torch, stream, lambda: h_keys.copy_(d_tmp, non_blocking=True), reps=3)
    # both directions at once (what the chunked host lookup needs)
    s_up, s_dn = torch.cuda.Stream(), torch.cuda.Stream()

    def both():
        s_up.wait_stream(stream)
        s_dn.wait_stream(stream)
        with torch.cuda.stream(s_up):
            d_tmp.copy_(h_keys, non_blocking=True)
        with torch.cuda.stream(s_dn):
            h_out.copy_(out, non_blocking=True)
        stream.wait_stream(s_up)
        stream.wait_stream(s_dn)
    bidir_ms = _timed(torch, stream, both, reps=3)
    del d_tmp
    link = {"h2d_GBps": 8 * n / (h2d_ms / 1e3) / 1e9, "d2h_GBps": 8 * n / (d2h_ms / 1e3) / 1e9,
            "both_directions_GBps": (8 * n + 8 * nq) / (bidir_ms / 1e3) / 1e9,
            "build_host_ms": c0.elapsed_time(c1), "lookup_host_ms": c1.elapsed_time(c2)}
    # the step cannot beat moving its bytes once over the link
    link["link_bound_ms"] = (16 * n / (link["h2d_GBps"] * 1e9) + max(8 * nq / (link["h2d_GBps"] * 1e9),
                                                                     9 * nq / (link["d2h_GBps"] * 1e9))) * 1e3

    # ---- roofline of the dominant kernel
    hbm, peak_kind = load_peaks()
    med = lambda xs: statistics.median(xs)
    lk = med(lookup_ms)
    pb = med([p[3] for p in part_ms])
    ne = med(nonempty)
    s_n = med(S)
    kernels = {
        "k_lookup_u64": {"ms": lk, "bytes": lookup_bytes_per_query(HIT, ne) * nq,
                         "model": f"{lookup_bytes_per_query(HIT, ne):.2f} B/query x {nq}"},
        "k_part_build": {"ms": pb, "bytes": part_build_bytes_per_key(s_n) * n,
                         "model": f"{part_build_bytes_per_key(s_n):.2f} B/key x {n}"},
    }
    two_level = part_ms[-1][5] == 2
    if two_level:
        # count A 8 + scatter A 16 read + 20 write + count B 4 + scatter B 20 read + 16 write
        kernels["grouping_2level"] = {"ms": med([p[4] for p in part_ms]), "bytes": 84.0 * n,
                                      "model": f"84 B/key x {n} (12 kernels)"}
    else:
        kernels["k_partition_scatter"] = {"ms": med([p[2] for p in part_ms]), "bytes": 32.0 * n,
                                          "model": f"32 B/key x {n}"}
        kernels["k_partition_count"] = {"ms": med([p[0] for p in part_ms]), "bytes": 8.0 * n,
                                        "model": f"8 B/key x {n}"}
    for k, v in kernels.items():
        v["GBps"] = v["bytes"] / (v["ms"] / 1e3) / 1e9
        v["frac"] = v["GBps"] / hbm
    # the dominant single kernel carries the roofline object
    dom = max(("k_lookup_u64", "k_part_build"), key=lambda k: kernels[k]["ms"])
    tr = kernel_traffic(dom, nq if dom == "k_lookup_u64" else n)
    D = kernels[dom]
    roofline = {"bound": "hbm", "achieved": D["GBps"], "peak": hbm, "unit": "GB/s",
                "frac": D["frac"], "traffic": tr, "kernel": dom, "peak_source": peak_kind,
                "bytes_model": D["model"]}

    line = {
        "metric": METRIC, "value": value, "unit": "keys+lookups/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_keys": n, "n_queries": nq, "hit_rate": HIT,
                   "values": "int64", "seed": SEED, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (512 MiB per array), no flush"},
        "build_keys_per_s": n * world / (med(build_ms) / 1e3),
        "lookups_per_s": nq * world / (lk / 1e3),
        "build_ms": med(build_ms), "lookup_ms": lk,
        "phases_ms": ({"grouping": med([p[4] for p in part_ms]), "part_build": pb} if two_level else
                      {"count": med([p[0] for p in part_ms]), "scan": med([p[1] for p in part_ms]),
                       "scatter": med([p[2] for p in part_ms]), "part_build": pb}),
        "S_over_n": s_n, "nonempty_frac": ne,
        "roofline": roofline,
        "kernels": {k: {"ms": round(v["ms"], 4), "GBps": round(v["GBps"], 1),
                        "frac": round(v["frac"], 4), "bytes_model": v["model"]}
                    for k, v in kernels.items()},
        "e2e": {"value": units / (e2e_ms / 1e3), "unit": "keys+lookups/s",
                "h2d_bytes_per_step": int(8 * n + 8 * n + 8 * nq),
                "d2h_bytes_per_step": int(8 * nq + nq), "ms_per_step": e2e_ms, "link": link},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "autotune": tune,
    }
    # ---- reference point: the search-based map (sort + binary search) on the same data
    if not args.no_search_baseline:
        sb, sl = [], []
        for i in range(4):
            a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a0.record(stream)
            sm = F.fks_sortmap_build(keys, vals)
            a1.record(stream)
            F.fks_sortmap_lookup(sm, queries, out, found, -1)
            a2.record(stream)
            torch.cuda.synchronize()
            if i >= 1:
                sb.append(a0.elapsed_time(a1))
                sl.append(a1.elapsed_time(a2))
            del sm
        assert np.array_equal(found.cpu().numpy(), w.expect_found)
        eb, el = [], []
        for i in range(4):
            a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a0.record(stream)
            em = F.fks_eytzmap_build(keys, vals)
            a1.record(stream)
            F.fks_sortmap_lookup(em, queries, out, found, -1)
            a2.record(stream)
            torch.cuda.synchronize()
            if i >= 1:
                eb.append(a0.elapsed_time(a1))
                el.append(a1.elapsed_time(a2))
            del em
        assert np.array_equal(found.cpu().numpy(), w.expect_found)
        assert np.array_equal(out.cpu().numpy(), np.where(w.expect_found == 1, w.expect_vals, -1))
        line["search_baseline"] = {
            "what": "GPU LSD radix sort of (key, value) + binary-search lookup, same data",
            "build_ms": med(sb), "lookup_ms": med(sl),
            "build_keys_per_s": n / (med(sb) / 1e3), "lookups_per_s": nq / (med(sl) / 1e3),
            "fks_speedup_build": med(sb) / med(build_ms), "fks_speedup_lookup": med(sl) / lk,
            "eytzinger": {"what": "the same sort, gathered into Eytzinger order; lookups descend the tree",
                          "build_ms": med(eb), "lookup_ms": med(el),
                          "lookups_per_s": nq / (med(el) / 1e3),
                          "fks_speedup_build": med(eb) / med(build_ms), "fks_speedup_lookup": med(el) / lk}}
    # ---- the other rows of the path: string keys, batched maps, recorded graphs, from_array
    if not args.no_extras:
        line["bucket_variants"] = run_bucket_variants(F, torch, hbm, keys, vals, queries, out, found, w, n, nq,
                                                      tune=not (args.no_autotune or args.tuning))
        line["inline_singletons"] = run_inline_singletons(F, torch, hbm, keys, vals, queries, out, found, w, n, nq)
        xs = args.extras_shift
        line["strings"] = run_strings(F, W, torch, hbm, xs)
        line["batched"] = run_batched(F, W, torch, hbm, xs)
        line["graph_builds"] = run_graph_builds(F, W, torch, xs)
        line["from_array"] = run_from_array(F, W, torch, hbm, xs)
        line["paper_table1"] = run_paper_table1(F, W, torch)
    # ---- serving stream: continuous batching against per-call launches
    if args.serve_requests > 0:
        line["serving"] = run_serving(args, F, W, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        with ctx.Pool(1) as pool:
            dt = pool.apply(cpu_sample_run, (args.cpu_sample, args.cpu_sample, SEED + 7))
        line["cpu_baseline"] = {"value": 2 * args.cpu_sample / dt, "unit": "keys+lookups/s",
                                "cores": 1, "kind": "oracle",
                                "sample": f"oracle build of {args.cpu_sample} keys + lookup of "
                                          f"{args.cpu_sample} queries (same generator), "
                                          f"{os.cpu_count()} host cores available"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
