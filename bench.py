"""Benchmark of the static bucketed hash table path on GB300.

Default workload: the HBM-bound BCHT configuration -- 2^28 unique uint32
key/value pairs, bucket of 16 pairs, three hash functions; each step builds a
table at load factor 0.99 and one at 0.9 (2.17 / 2.39 GB, far beyond L2) and
runs 2^28 all-positive and 2^28 all-negative finds on each. ``value`` is the
keys processed per second (built + queried), device-timed with inputs
resident in HBM; ``e2e`` is the same metric through the public API from
pinned host buffers (copies inside the timed region).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank builds and queries its own independent tables
(weak scaling, no data-path collective).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gkeys/s build and find (pos/neg) at LF 0.9/0.99, % HBM peak; served p99 latency"
LFS = (0.99, 0.9)
SEED = 0x6768740003  # input seed of the HBM-bound BCHT configuration


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--log2n", type=int, default=28, help="keys per table (log2)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ceilings", action="store_true", help="skip the memory-pattern ceiling probe")
    ap.add_argument("--no-served", action="store_true", help="skip the served-pool record of the default line")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-tables record of the default line")
    ap.add_argument("--tile-lanes", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--build-tile-lanes", type=int, default=0)
    ap.add_argument("--keys-per-lane", type=int, default=0, help="find: query sets in flight per lane")
    ap.add_argument("--build-keys-per-lane", type=int, default=0, help="insert: keys in flight per lane")
    ap.add_argument("--find-async", type=int, default=0, choices=[-1, 0, 1])
    ap.add_argument("--find-grouped", type=int, default=0, choices=[-1, 0, 1],
                    help="grouped find (rounds by table range, opt-in): 1 on, else per query")
    ap.add_argument("--group-build", type=int, default=0, choices=[-1, 0, 1],
                    help="1: group the pairs by first-choice bucket range before the build")
    ap.add_argument("--ranked-build", type=int, default=0, choices=[-1, 0],
                    help="BCHT build: 0 two-phase (ranked first-choice placement, then cuckoo insert), "
                         "-1 cuckoo insert of every key")
    ap.add_argument("--workload", choices=["hbm", "batched", "served", "sweep", "success", "sizes"], default="hbm",
                    help="hbm: 2^28-key BCHT tables (default); batched: 512 uneven tables in one graph "
                         "launch; served: a table pool under Poisson request arrivals")
    ap.add_argument("--served-seconds", type=float, default=1.0, help="served: length of the arrival trace")
    ap.add_argument("--sharded", action="store_true",
                    help="one table sharded over the ranks (partition hash + all-to-all) instead of a table per rank")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(base: int, rank: int) -> int:
    """Input seed of a rank: every rank builds and queries its own tables."""
    return base + rank


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of a per-rank value over all ranks (identity on one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(keys_per_rank_step: int, steps: int, world: int, max_ms: float) -> float:
    """Gkeys/s of the whole job: every rank's keys over the slowest rank's time."""
    return world * keys_per_rank_step * steps / (max_ms / 1e3) / 1e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the find
# kernel, averaged over its four launches of one step of the default workload:
# one-pass ncu metrics over the recorded step of `bench.py --steps 1 --warmup 1`
# at 2^28 keys. It describes the kernel source it was captured from,
# identified by a hash of the find kernel's headers; after any change to them
# the traffic is reported as null.
FIND_TRAFFIC = {"bytes_per_launch": 60460572544, "source_sha256_16": "d0a797b09e952b68",
               "kernel": "bcht_find_async_kernel"}


def build_kernels(st: dict) -> list[str]:
    """The library kernels one build attempt launches, from the table's stats."""
    if st["last_build_split"]:  # two grouping levels, block placement, no fill
        return ["region_cursors_kernel", "group_scatter_kernel", "region_cursors_kernel", "group_scatter_kernel",
                "block_place_kernel", "bucketed_insert_kernel"]
    ks = ["fill_kernel"]
    if st["last_build_grouped"]:  # per-group regions when placed by rank, else a count pass and prefix
        ks += (["region_cursors_kernel"] if st["last_build_ranked"] else ["group_count_kernel", "group_scan_kernel"])
        ks += ["group_scatter_kernel"]
    if st["last_build_ranked"]:
        ks += ["rank_place_kernel"]
    return ks + ["bucketed_insert_kernel"]


def find_kernels(st: dict) -> list[str]:
    """The library kernels one find launches, from the table's stats."""
    if st["last_find_grouped"]:  # per round: two groupings and the lookup; then the return to query order
        rnd = ["region_cursors_kernel", "group_scatter_kernel", "region_cursors_kernel", "group_scatter_kernel",
               "grouped_lookup_kernel"]
        return rnd * st["num_hashes"] + ["grouped_spill_kernel"] + ["region_cursors_kernel", "group_scatter_kernel"] * 2 \
            + ["window_write_kernel"]
    return ["bcht_find_async_kernel" if st["find_staged"] else "bucketed_find_kernel"]


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("ght_find.cuh", "ght_find_async.cuh", "ght_device.cuh"):
        with open(os.path.join(ROOT, "paper_2108_07232_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def bytes_per_key(op: str, p: float, lf: float) -> float:
    """Algorithmic bytes per key (query/result or pair, 128 B per bucket probe,
    plus one write-back of the table for inserts)."""
    if op == "find":
        return 4 + 4 + 128 * p
    if op == "insert":
        return 8 + 128 * p + 8 / lf
    if op == "fill":
        return 8 / lf
    raise ValueError(op)


PROBE_MODES = {0: "random_line_read", 1: "line_read_then_cas", 2: "line_read_then_cas_waited", 3: "atomic_add_only",
               4: "random_half_line_read", 5: "half_line_then_dependent_sector"}


def measure_ceilings(num_lines: int, ops: int, dev, reps: int = 3) -> dict:
    """Rates of the tables' memory access patterns on random 128-byte lines of
    a buffer as large as the table (ght_probe_lines), untimed by the step."""
    import torch

    import paper_2108_07232_gb300 as G
    buf = torch.empty(num_lines * 128 // 8, dtype=torch.int64, device=dev)
    buf.fill_(-1)
    stream = torch.cuda.current_stream(dev).cuda_stream
    out = {}
    for mode, name in PROBE_MODES.items():
        G.ght_probe_lines(mode, buf, num_lines, ops, 7, stream)  # warm
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(reps):
            G.ght_probe_lines(mode, buf, num_lines, ops, 11 + r, stream)
        e1.record()
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        out[name] = {"glines_s": round(ops / sec / 1e9, 2), "ms": round(sec * 1e3, 3),
                     "line_gbs": round(128 * ops / sec / 1e9, 1)}
    del buf
    torch.cuda.empty_cache()
    out["note"] = (f"{ops} operations on random lines of a {num_lines * 128 / 1e9:.2f} GB buffer; line_gbs counts "
                   "128 B per operation (the atomic-only mode touches 8 B)")
    return out


# ------------------------------------------------------------- CPU oracle ---

def oracle_sample(n: int, lfs=LFS):
    """Time the oracle (as it stands, single-threaded) on n keys per load factor:
    build, then n positive and n negative finds. Returns (keys, seconds)."""
    import oracle as O
    import workloads as W
    keys, vals = W.make_keys(n, SEED), W.make_values(n, SEED)
    pos = W.make_queries(keys, n, 1.0, SEED)
    neg = W.make_negatives(n, n, SEED)
    k, v, qp, qn = O._u32(keys), O._u32(vals), O._u32(pos), O._u32(neg)
    total, secs = 0, 0.0
    for lf in lfs:
        T = O.Table(O.BCHT, n, lf, seed=SEED)
        t0 = time.perf_counter()
        ok = T.build(k, v)
        T.find(qp)
        T.find(qn)
        secs += time.perf_counter() - t0
        if ok != 1:
            raise RuntimeError("oracle build failed")
        total += 3 * n
    return total, secs


def run_reference(args, world, rank):
    if rank != 0:
        return
    n = 1 << 21
    oracle_sample(1 << 12)  # compile / warm
    for _ in range(args.warmup):
        oracle_sample(n)
    keys = secs = 0
    for _ in range(args.steps):
        k, s = oracle_sample(n)
        keys += k
        secs += s
    value = keys / secs / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config_of(args, sample_n=n), "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                         "sample": f"BCHT b=16 h=3, {n} keys per load factor {list(LFS)}: build + "
                                   f"{n} positive + {n} negative finds, sequential C oracle"},
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(args, sample_n=None):
    c = {"workload": f"bcht_b16_h3_n2^{args.log2n}_lf0.99+0.9_find_pos+neg",
         "scheme": "BCHT", "bucket_size": 16, "num_hashes": 3, "keys_per_table": 1 << args.log2n,
         "load_factors": list(LFS), "queries_per_table": 2 << args.log2n, "positive_fractions": [1.0, 0.0],
         "l2": "inputs larger than L2 (tables 2.2-2.4 GB, key arrays 1 GB)", "input_seed": SEED}
    if sample_n:
        c["oracle_sample_keys"] = sample_n
    return c


# ------------------------------------------------------------------- ours ---

def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    import paper_2108_07232_gb300 as G
    import workloads as W
    from paper_2108_07232_gb300 import build as B

    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or not os.path.exists(G.lib_path()):
        B.build()
    if world > 1:
        dist.barrier()
    n = 1 << args.log2n
    seed = rank_seed(SEED, rank)
    keys = W.make_keys(n, seed, device=dev)
    vals = W.make_values(n, seed, device=dev)
    pos = W.make_queries(keys, n, 1.0, seed)
    neg = W.make_negatives(n, n, seed, device=dev)
    out = torch.empty_like(keys)
    cfg = {}
    if args.tile_lanes:
        cfg["tile_lanes"] = args.tile_lanes
    if args.blocks_per_sm:
        cfg["blocks_per_sm"] = args.blocks_per_sm
    if args.build_tile_lanes:
        cfg["build_tile_lanes"] = args.build_tile_lanes
    if args.ranked_build:
        cfg["ranked_build"] = args.ranked_build
    if args.group_build:
        cfg["group_build"] = args.group_build
    if args.keys_per_lane:
        cfg["keys_per_lane"] = args.keys_per_lane
    if args.build_keys_per_lane:
        cfg["build_keys_per_lane"] = args.build_keys_per_lane
    if args.find_async:
        cfg["find_async"] = args.find_async
    if args.find_grouped:
        cfg["find_grouped"] = args.find_grouped
    tables = {lf: G.HashTable("bcht", n, lf, seed=seed, **cfg) for lf in LFS}
    torch.cuda.synchronize()

    launches = [0]
    phase_ms = {f"{op}@{lf}": [] for lf in LFS
                for op in ("fill", "group", "split", "place", "insert", "find_pos", "find_neg")}

    def step(record: bool):
        for lf in LFS:
            t = tables[lf]
            t.build(keys, vals)
            st = t.stats()
            launches[0] += len(build_kernels(st)) * st["attempts"]
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record()
            t.find(pos, out)
            e1.record()
            t.find(neg, out)
            e2.record()
            launches[0] += 2 * len(find_kernels(t.stats()))
            if record:
                phase_ms[f"fill@{lf}"].append(st["last_fill_ms"])
                phase_ms[f"group@{lf}"].append(max(st["last_group_ms"], 0.0))
                phase_ms[f"split@{lf}"].append(max(st["last_split_ms"], 0.0))
                phase_ms[f"place@{lf}"].append(max(st["last_place_ms"], 0.0))
                phase_ms[f"insert@{lf}"].append(st["last_insert_ms"])
                e2.synchronize()
                phase_ms[f"find_pos@{lf}"].append(e0.elapsed_time(e1))
                phase_ms[f"find_neg@{lf}"].append(e1.elapsed_time(e2))

    for _ in range(args.warmup):
        step(False)
    # kernel phase times (one separate, recorded pass; the timed loop below has no extra syncs)
    step(True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    launches[0] = 0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step(False)
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = reduce_max(ev0.elapsed_time(ev1), world, dev)
    keys_per_step = len(LFS) * 3 * n
    value = whole_job_value(keys_per_step, args.steps, world, ms)
    gpu_launches = launches[0]
    # the device build's kernels, read before the end-to-end leg rebuilds the
    # tables from host buffers (a different build path)
    st_dev = tables[LFS[0]].stats()

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        # page-locked host buffers allocated as such and filled from the
        # device (no pageable intermediate copies)
        def pinned_copy(x):
            h = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
            h.copy_(x)
            return h

        hk, hv = pinned_copy(keys), pinned_copy(vals)
        hp, hn = pinned_copy(pos), pinned_copy(neg)
        hout = torch.empty(hk.shape, dtype=hk.dtype, pin_memory=True)

        call_ms = {f"{op}@{lf}": [] for lf in LFS for op in ("build", "find_pos", "find_neg")}
        h2d_gbs = {k: [] for k in call_ms}

        def host_step():
            # each call returns once its results are on the host, so the wall
            # time of each is its end-to-end time
            for lf in LFS:
                t = tables[lf]
                for op, fn in (("build", lambda: t.build(hk, hv)), ("find_pos", lambda: t.find(hp, hout)),
                               ("find_neg", lambda: t.find(hn, hout))):
                    c0 = time.perf_counter()
                    fn()
                    call_ms[f"{op}@{lf}"].append(1e3 * (time.perf_counter() - c0))
                    s = t.stats()  # host-to-device copy span of that call (device events)
                    if s["last_h2d_ms"] > 0:
                        h2d_gbs[f"{op}@{lf}"].append(s["last_h2d_bytes"] / (s["last_h2d_ms"] / 1e3) / 1e9)
            return int(hout[0])  # the step's result is on the host

        for _ in range(max(1, args.warmup)):
            host_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        step_ms = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s0 = time.perf_counter()
            host_step()
            step_ms.append(round(1e3 * (time.perf_counter() - s0), 2))
        torch.cuda.synchronize()
        el = reduce_max(time.perf_counter() - t0, world, dev)
        e2e = {"value": whole_job_value(keys_per_step, args.steps, world, 1e3 * el), "unit": "Gkeys/s",
               "h2d_bytes_per_step": len(LFS) * (8 * n + 8 * n),
               "d2h_bytes_per_step": len(LFS) * 8 * n,
               "api": "HashTable.build/find on pinned CPU tensors (ght_build_host: the insert reads the pinned "
                      "pairs in place; ght_find_host: pipelined chunk copies in and out)",
               "step_ms": step_ms,
               "call_ms": {k: round(statistics.median(v), 3) for k, v in call_ms.items()},
               "call_ms_max": {k: round(max(v), 3) for k, v in call_ms.items()},
               "h2d_gbs_median_min": {k: [round(statistics.median(v), 1), round(min(v), 1)]
                                      for k, v in h2d_gbs.items() if v}}

    # probe counts for the algorithmic bytes: one extra counted build/find (untimed)
    probes = {}
    for lf in LFS:
        tc = G.HashTable("bcht", n, lf, seed=seed, count_probes=1, **cfg)
        tc.build(keys, vals)
        st = tc.stats()
        p_ins = st["insert_probes"] / n
        tc.reset_counters()
        tc.find(pos, out)
        p_pos = tc.stats()["find_probes"] / n
        tc.reset_counters()
        tc.find(neg, out)
        p_neg = tc.stats()["find_probes"] / n
        probes[lf] = {"insert": p_ins, "find_pos": p_pos, "find_neg": p_neg,
                      "insert_retries": st["insert_retries"] / n}
        del tc

    peak, peak_src = peaks()
    kernels = {}
    st0 = st_dev
    bks = build_kernels(st0)
    has_fill = "fill_kernel" in bks  # else the placement writes every line: no fill to rate
    find_name = "+".join(dict.fromkeys(find_kernels(st0)))
    for lf in LFS:
        # a build's work after the fill: the grouping (one or two levels) and
        # the ranked placement (when the build does them) and the cuckoo
        # insert, timed together
        phase_ms[f"build@{lf}"] = [a + b + c + d for a, b, c, d in
                                   zip(phase_ms[f"group@{lf}"], phase_ms[f"split@{lf}"], phase_ms[f"place@{lf}"],
                                       phase_ms[f"insert@{lf}"])]
        for op, key, pp in ((("fill", "fill", 0.0),) if has_fill else ()) + (
                ("insert", "build", probes[lf]["insert"]), ("find", "find_pos", probes[lf]["find_pos"]),
                ("find", "find_neg", probes[lf]["find_neg"])):
            t_ms = statistics.median(phase_ms[f"{key}@{lf}"])
            bpk = bytes_per_key(op, pp, lf)
            gbs = bpk * n / (t_ms / 1e3) / 1e9
            kernels[f"{key}@{lf}"] = {"ms": round(t_ms, 4), "gkeys_s": round(n / (t_ms / 1e3) / 1e9, 3),
                                      "bytes_per_key": round(bpk, 2), "achieved_gbs": round(gbs, 1),
                                      "frac_of_hbm": round(gbs / peak, 4)}
    # dominant kernel = the kernel function with the most device time per step
    build_name = "+".join(dict.fromkeys(k for k in bks if k != "fill_kernel"))
    funcs = {find_name: [k for k in kernels if k.startswith("find")],
             build_name: [k for k in kernels if k.startswith("build")]}
    if has_fill:
        funcs["fill_kernel"] = [k for k in kernels if k.startswith("fill")]
    per_func = {}
    for f, ks in funcs.items():
        t_ms = sum(kernels[k]["ms"] for k in ks)
        byts = sum(kernels[k]["bytes_per_key"] * n for k in ks)
        per_func[f] = {"launches_per_step": len(ks), "ms_per_step": round(t_ms, 3),
                       "achieved_gbs": round(byts / (t_ms / 1e3) / 1e9, 1),
                       "frac_of_hbm": round(byts / (t_ms / 1e3) / 1e9 / peak, 4)}
    dom_name = max(per_func, key=lambda f: per_func[f]["ms_per_step"])
    dom = per_func[dom_name]
    traffic = None
    if (dom_name == FIND_TRAFFIC.get("kernel", "bucketed_find_kernel") and args.log2n == 28
            and kernel_source_hash() == FIND_TRAFFIC["source_sha256_16"]):
        traffic = FIND_TRAFFIC["bytes_per_launch"]
    alg_per_launch = sum(kernels[k]["bytes_per_key"] * n for k in funcs[dom_name]) / len(funcs[dom_name])
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": dom["achieved_gbs"], "peak": peak,
                "unit": "GB/s", "frac": dom["frac_of_hbm"], "traffic": traffic,
                "algorithmic_bytes_per_launch": round(alg_per_launch),
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s",
                "note": "achieved = algorithmic bytes of the kernel's launches in one step / their summed CUDA-event time"}

    ceilings = None
    if not args.no_ceilings:
        ceilings = measure_ceilings(tables[LFS[0]].stats()["num_buckets"], n, dev)
        ins_lines = sum(probes[lf]["insert"] * n for lf in LFS) / sum(kernels[f"build@{lf}"]["ms"] / 1e3 for lf in LFS)
        find_lines = (sum((probes[lf]["find_pos"] + probes[lf]["find_neg"]) * n for lf in LFS)
                      / sum((kernels[f"find_pos@{lf}"]["ms"] + kernels[f"find_neg@{lf}"]["ms"]) / 1e3 for lf in LFS))
        ceilings["kernels_glines_s"] = {"find": round(find_lines / 1e9, 2), "insert": round(ins_lines / 1e9, 2)}

    # the metric's served-latency clause and the batched path, measured on a
    # smaller scale beside the headline (rank 0 of a one-GPU run)
    served = batched = None
    if rank == 0 and world == 1 and not args.no_served:
        served = served_measure(dev, SEED + 2, 64, 22, 0.3, build_log2=(20, 22))
    if rank == 0 and world == 1 and not args.no_batched:
        batched = batched_measure(dev, SEED + 1, 512, 20, 3, 2)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns = 1 << 22
        keys_done, secs = oracle_sample(ns)
        cpu = {"value": keys_done / secs / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
               "sample": f"BCHT b=16 h=3, {ns} keys per load factor {list(LFS)}: sequential C oracle "
                         f"build + {ns} positive + {ns} negative finds ({secs:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gkeys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": config_of(args), "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches, "clocks": clocks,
            "kernels": kernels, "kernel_functions": per_func, "probes_per_key": probes,
            "build_phases_ms": {str(lf): {ph: round(statistics.median(phase_ms[f"{ph}@{lf}"]), 4)
                                         for ph in ("fill", "group", "split", "place", "insert")} for lf in LFS},
            "pattern_ceilings": ceilings, "served": served, "batched": batched,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_sharded(args, world, rank, local):
    """One table sharded over the ranks (paper_2108_07232_gb300.sharded): each
    rank holds 2^log2n pairs and queries of its own; per step a table of all
    ranks' pairs is built at LF 0.99 and at 0.9 (partition by the partition
    hash, all-to-all, shard build) and each rank's 2^log2n positive and
    2^log2n negative queries are found (partition, all-to-all, shard find,
    reverse all-to-all, return to query order). Weak scaling: per-rank work is
    fixed as ranks are added."""
    import torch
    import torch.distributed as dist

    import workloads as W
    from paper_2108_07232_gb300 import build as B
    from paper_2108_07232_gb300.sharded import ShardedTable

    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if world > 1:
        dist.barrier()
    n = 1 << args.log2n
    seed = rank_seed(SEED, rank)
    keys = W.make_keys(n, seed, device=dev)
    vals = W.make_values(n, seed, device=dev)
    pos = W.make_queries(keys, n, 1.0, seed)
    neg = W.make_negatives(n, n, seed, device=dev)
    tables = {lf: ShardedTable("bcht", world * n, lf, seed=SEED) for lf in LFS}

    def step():
        for lf in LFS:
            t = tables[lf]
            t.build(keys, vals)
            t.find(pos)
            t.find(neg)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = reduce_max(ev0.elapsed_time(ev1), world, dev)
    value = whole_job_value(len(LFS) * 3 * n, args.steps, world, ms)
    shard = {str(lf): tables[lf].n_local for lf in LFS}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": round(value, 3), "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"bcht_b16_h3_sharded_one_table_{world}x2^{args.log2n}_lf0.99+0.9_find_pos+neg",
                       "keys_per_rank": n, "load_factors": list(LFS), "exchange": "nccl all-to-all" if world > 1 else
                       "none (one rank: partition and the local shard only)",
                       "l2": "inputs larger than L2", "input_seed": SEED},
            "shard_keys_rank0": shard, "clocks": clocks,
        }), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def batched_measure(dev, seed, num_tables, log2_max, steps, warmup):
    """Independent BCHT tables, key counts floor(2^(10 + (log2_max - 10) u)),
    LF ~ U[0.8, 0.99], 2 queries per key (50 % positive): one autotuned
    CUDA-graph launch per step (build + find of every table) against the same
    tables built and queried with one plain build and one find call each."""
    import torch

    import paper_2108_07232_gb300 as G
    import workloads as W

    wk = W.make_batch(num_tables, 10, log2_max, 0.8, 0.99, 2.0, 0.5, seed, device=dev)
    k, v, q = wk["keys"], wk["values"], wk["queries"]
    ko, qo = wk["key_offsets"], wk["query_offsets"]
    out = torch.empty_like(q)
    b = G.Batch(wk["capacities"], wk["load_factors"], seed=seed)
    b.set_layout(ko, qo)
    tuned = b.autotune(k, v, q, out)
    items = int(ko[-1]) + int(qo[-1])

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(warmup):
        b.run(k, v, q, out)
    ms_batched = timed(lambda: b.run(k, v, q, out), steps)
    graph_ms = b.stats()["last_run_ms"]
    ref = out.clone()
    # plain: one table object per table, one build and one find call each
    tables = [G.HashTable("bcht", int(wk["capacities"][t]), float(wk["load_factors"][t]), seed=seed + t)
              for t in range(num_tables)]
    sl = [(int(ko[t]), int(ko[t + 1]), int(qo[t]), int(qo[t + 1])) for t in range(num_tables)]

    def plain():
        for t, (a0, a1, q0, q1) in zip(tables, sl):
            t.build(k[a0:a1], v[a0:a1])
            t.find(q[q0:q1], out[q0:q1])

    for _ in range(warmup):
        plain()
    ms_plain = timed(plain, steps)
    same = bool(torch.equal(out, ref))
    st = b.stats()
    b.close()
    return {
        "value": round(items * steps / (ms_batched / 1e3) / 1e9, 3), "unit": "Gkeys/s",
        "ms_per_step": round(ms_batched / steps, 3), "steps": steps, "warmup": warmup,
        "config": {"workload": f"batched_{num_tables}_bcht_n2^10..2^{log2_max}_lf0.8..0.99_q2x_f0.5",
                   "tables": num_tables, "total_keys": int(ko[-1]), "total_queries": int(qo[-1]),
                   "input_seed": seed},
        "graph_ms": graph_ms, "autotuned": {kk: tuned[kk] for kk in ("tile_lanes", "keys_per_lane", "blocks_per_sm",
                                                                     "build_tile_lanes", "build_keys_per_lane",
                                                                     "build_blocks_per_sm") if kk in tuned},
        "rebuilds": st["rebuilds"],
        "plain_back_to_back": {"value": round(items * steps / (ms_plain / 1e3) / 1e9, 3), "unit": "Gkeys/s",
                               "ms_per_step": round(ms_plain / steps, 3),
                               "launches_per_step": num_tables * 3, "host_syncs_per_step": num_tables},
        "speedup_vs_plain": round(ms_plain / ms_batched, 3), "results_identical": same,
    }


def run_batched(args, world, rank, local):
    """512 independent BCHT tables of 2^10..2^22 keys in one graph launch per
    step against back-to-back plain calls (see batched_measure)."""
    import torch

    from paper_2108_07232_gb300 import build as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    r = batched_measure(dev, SEED + 1 + rank, 512, 22, args.steps, args.warmup)
    line = {
        "metric": "Gkeys/s batched build+find, 512 BCHT tables in one graph launch", "value": r.pop("value"),
        "unit": r.pop("unit"), "n_gpus": 1, "steps": r.pop("steps"), "warmup": r.pop("warmup"),
        "ms_per_step": r.pop("ms_per_step"), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": r.pop("config"), **r,
    }
    print(json.dumps(line), flush=True)


def served_measure(dev, seed, num_tables, log2_max, seconds, build_log2=(20, 24), budget=60 << 30):
    """num_tables resident BCHT tables of 2^16..2^log2_max keys (log-uniform) at
    LF 0.95 in a pool with an HBM budget. A Poisson stream of find batches
    (sizes log-uniform in [1, 2^20], 70 % positive keys) at 80 % of the pool's
    measured capacity, plus a build request of a new 2^build_log2[0]..
    2^build_log2[1]-key table every 100 ms, is replayed through the pool
    (continuous batching) and as serial plain calls; p50/p99 latency and
    aggregate throughput of both, and whether every answer is the same."""
    import numpy as np
    import torch

    import paper_2108_07232_gb300 as G
    import workloads as W

    rng = np.random.default_rng(seed)
    pool = G.Pool(budget, device=dev)
    span_log2 = log2_max - 16
    sizes = [int(2 ** (16 + span_log2 * W.uniform01(t, seed))) for t in range(num_tables)]
    qpool, ids = [], []
    for t, n in enumerate(sizes):
        k, v = W.make_keys(n, seed + t, device=dev), W.make_values(n, seed + t, device=dev)
        tk, tid = pool.submit_build(n, 0.95, seed + t, k, v)
        pool.wait(tk, timeout=600)
        ids.append(tid)
        qpool.append(W.make_queries(k, 1 << 20, 0.7, seed + 1000 + t))
        del k, v

    def make_trace(count, rate):
        arr = np.cumsum(rng.exponential(1.0 / rate, count)) if rate else np.zeros(count)
        tr = []
        for i in range(count):
            t = int(rng.integers(0, num_tables))
            size = int(2 ** rng.uniform(0, 20))
            off = int(rng.integers(0, (1 << 20) - size + 1))
            q = qpool[t][off:off + size]
            tr.append({"kind": "find", "table": ids[t], "queries": q, "out": torch.empty_like(q),
                       "arrival_s": float(arr[i])})
        return tr

    # capacity: a burst of requests all arriving at once
    burst = make_trace(2000, 0)
    pool.replay(burst)
    _, _, mk = pool.replay(burst)
    burst_q = sum(t["queries"].numel() for t in burst)
    capacity_qps = burst_q / mk
    mean_size = burst_q / len(burst)
    rate = 0.8 * capacity_qps / mean_size
    count = max(100, int(rate * seconds))
    trace = make_trace(count, rate)
    span = trace[-1]["arrival_s"]
    n_builds = int(span / 0.1)
    builds = []
    b_lo, b_hi = build_log2
    for j in range(n_builds):
        n = int(2 ** (b_lo + (b_hi - b_lo) * W.uniform01(j, seed ^ 0x62)))
        k, v = W.make_keys(n, seed + 5000 + j, device=dev), W.make_values(n, seed + 5000 + j, device=dev)
        builds.append({"kind": "build", "keys": k, "values": v, "capacity": n, "load_factor": 0.95,
                       "seed": seed + 5000 + j, "arrival_s": 0.1 * (j + 1)})
    full = sorted(trace + builds, key=lambda r: r["arrival_s"])
    out = {}
    for mode in ("pool", "serial"):
        for r in full:
            if r["kind"] == "find":
                r["out"] = torch.empty_like(r["queries"])
        lat, st, mk = pool.replay(full, serial=(mode == "serial"))
        fl = np.array([lat[i] for i, r in enumerate(full) if r["kind"] == "find"])
        keys_done = sum(r["queries"].numel() if r["kind"] == "find" else r["keys"].numel() for r in full)
        out[mode] = {"p50_ms": round(1e3 * float(np.percentile(fl, 50)), 3),
                     "p99_ms": round(1e3 * float(np.percentile(fl, 99)), 3),
                     "gkeys_s": round(keys_done / mk / 1e9, 3), "makespan_s": round(mk, 4),
                     "ok": bool((st == 0).all()),
                     "outs": [r["out"] for r in full if r["kind"] == "find"]}
    same = all(torch.equal(a, b) for a, b in zip(out["pool"].pop("outs"), out["serial"].pop("outs")))
    st = pool.stats()
    pool.close()
    return {
        "config": {"workload": f"served_{num_tables}_bcht_n2^16..2^{log2_max}_lf0.95_budget{budget >> 30}GB",
                   "find_requests": count, "build_requests": n_builds,
                   "build_keys": f"2^{b_lo}..2^{b_hi} every 100 ms", "arrival_rate_per_s": round(rate, 1),
                   "trace_s": round(span, 3), "offered_load": "0.8 x measured capacity",
                   "mean_find_size": round(mean_size, 1), "input_seed": seed},
        "capacity_gqueries_s": round(capacity_qps / 1e9, 3), "pool": out["pool"], "serial_plain_calls": out["serial"],
        "results_identical": same, "mean_requests_per_launch": round(st["mean_requests_per_launch"], 2),
    }


def run_served(args, world, rank, local):
    """128 resident tables of 2^16..2^24 keys under a Poisson request stream
    (see served_measure)."""
    import torch

    from paper_2108_07232_gb300 import build as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    r = served_measure(dev, SEED + 2 + rank, 128, 24, args.served_seconds)
    line = {
        "metric": "served p50/p99 find latency and Gkeys/s, 128 resident BCHT tables, continuous batching",
        "value": r["pool"]["p99_ms"], "unit": "ms (p99 find latency)", "n_gpus": 1, "steps": 1, "warmup": 1,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        **r,
    }
    print(json.dumps(line), flush=True)


PAPER_IHT_THRESHOLD = {  # (b, t): (insert, positive find) probes at LF 0.86 printed in Sec. VII-A3
    (16, 4): (2.68, 2.11), (16, 7): (2.29, 1.86), (16, 10): (1.89, 1.6), (16, 13): (1.49, 1.33),
}

PAPER_PROBES = {  # (scheme, lf): (insert, find_pos, find_neg) printed in Sec. VII (50M keys, TITAN V)
    ("bcht", 0.9): (1.11, None, None), ("bcht", 0.99): (1.43, 1.38, 2.80),
    ("p2bht", 0.8): (2.0, 1.33, 2.0), ("iht", 0.86): (1.49, 1.33, 3.0),
}


def _time_ms(fn, reps=5):
    import torch
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def measure_table(scheme, n, lf, fracs, seed, dev, **cfg):
    """Build and find throughput (Gkeys/s, CUDA events, median of reps) and probe
    counts of one table configuration on synthetic keys."""
    import torch

    import paper_2108_07232_gb300 as G
    import workloads as W

    keys, vals = W.make_keys(n, seed, device=dev), W.make_values(n, seed, device=dev)
    negs = W.make_negatives(n, n, seed, device=dev)
    qs = {f: W.make_queries(keys, n, f, seed, negs) for f in fracs}
    out = torch.empty_like(keys)
    t = G.HashTable(scheme, n, lf, seed=seed, max_attempts=3, **cfg)
    try:
        t.build(keys, vals)
    except G.GhtError as e:
        return {"scheme": scheme, "n": n, "lf": lf, **cfg, "built": False, "status": e.status}
    build_ms = _time_ms(lambda: t.build(keys, vals))
    r = {"scheme": scheme, "n": n, "lf": lf, **cfg, "built": True,
         "build_gkeys_s": round(n / build_ms / 1e6, 3)}
    for f in fracs:
        ms = _time_ms(lambda: t.find(qs[f], out))
        r[f"find_gkeys_s_f{f}"] = round(n / ms / 1e6, 3)
    tc = G.HashTable(scheme, n, lf, seed=seed, max_attempts=3, count_probes=1, **cfg)
    tc.build(keys, vals)
    r["insert_probes"] = round(tc.stats()["insert_probes"] / n, 4)
    for f in fracs:
        tc.reset_counters()
        tc.find(qs[f], out)
        r[f"find_probes_f{f}"] = round(tc.stats()["find_probes"] / n, 4)
    if (scheme, lf) in PAPER_PROBES:
        r["paper_probes_insert_pos_neg"] = PAPER_PROBES[(scheme, lf)]
    return r


def run_sweep(args, world, rank, local):
    """The L2-resident case (BCHT, 2^20 keys, LF 0.9, 2^20 queries at 50 %
    positive) and the scheme sweep at 2^24 keys (BCHT, P2BHT, IHT, 1CHT with
    3 and 4 hash functions; LF 0.6..0.99; positive fraction 0, 0.5, 1): build and
    find throughput per combination, probes per key, and build failures where a
    scheme cannot reach the load factor (expected, Sec. VII-A)."""
    import torch

    import paper_2108_07232_gb300 as G
    import workloads as W
    from paper_2108_07232_gb300 import build as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    rows = []

    rows.append({"config": "bcht_n2^20_lf0.9_f0.5 (L2-resident)",
                 **measure_table("bcht", 1 << 20, 0.9, (0.5,), SEED + 10, dev)})
    n = 1 << 24
    for scheme, cfg in (("bcht", {}), ("p2bht", {}), ("iht", {}), ("cuckoo1", {}), ("cuckoo1", {"num_hashes": 4})):
        for lf in (0.6, 0.8, 0.9, 0.95, 0.99):
            rows.append({"config": "scheme_sweep_n2^24", **measure_table(scheme, n, lf, (0.0, 0.5, 1.0), SEED + 11, dev, **cfg)})
    for scheme, lf in (("p2bht", 0.86), ("iht", 0.86), ("bcht_lb", 0.9), ("bcht_lb", 0.99)):
        rows.append({"config": "paper_points_n2^24", **measure_table(scheme, n, lf, (0.0, 1.0), SEED + 12, dev)})
    for scheme, cfg, lf in (("p2bht", {"bucket_size": 32}, 0.9), ("iht", {"bucket_size": 32}, 0.9)):
        rows.append({"config": "b32_n2^24", **measure_table(scheme, n, lf, (0.0, 1.0), SEED + 13, dev, **cfg)})
    for lf in (0.9, 0.99):
        rows.append({"config": "keys_only_set_n2^24", **measure_table("bcht_set", n, lf, (0.0, 0.5, 1.0), SEED + 14, dev)})
    # Sec. VII-A3: IHT thresholds at 20/40/60/80 % of b (t = 4, 7, 10, 13 for
    # b = 16 at LF 0.86, where the paper prints insert and positive-find
    # probes; t = 7, 13, 20, 26 for b = 32 at LF 0.9)
    for b, lf, ts in ((16, 0.86, (4, 7, 10, 13)), (32, 0.9, (7, 13, 20, 26))):
        for t in ts:
            r = measure_table("iht", n, lf, (0.0, 1.0), SEED + 15, dev, bucket_size=b, threshold=t)
            if (b, t) in PAPER_IHT_THRESHOLD:
                r["paper_probes_insert_pos"] = PAPER_IHT_THRESHOLD[(b, t)]
            rows.append({"config": "iht_threshold_sweep_n2^24", **r})
    print(json.dumps({"metric": "scheme sweep: build/find Gkeys/s and probes per key", "workload": "sweep",
                      "rows": rows}), flush=True)


def run_sizes(args, world, rank, local):
    """Throughput against table size at fixed load factors (the paper's
    Sec. VII-A size sweeps): BCHT at LF 0.8 and 0.9, P2BHT, IHT and 1CHT at 0.8,
    P2BHT and IHT with 32-slot buckets at 0.9; 2^16 to 2^26 keys (BCHT to
    2^28); build, and find at 50 % positive. Small tables are L2-resident."""
    import torch

    from paper_2108_07232_gb300 import build as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    rows = []
    cases = [("bcht", 0.8, {}, 28), ("bcht", 0.9, {}, 28), ("p2bht", 0.8, {}, 26), ("iht", 0.8, {}, 26),
             ("cuckoo1", 0.8, {}, 26), ("p2bht", 0.9, {"bucket_size": 32}, 26), ("iht", 0.9, {"bucket_size": 32}, 26)]
    for scheme, lf, cfg, top in cases:
        for lg in range(16, top + 1, 2):
            r = measure_table(scheme, 1 << lg, lf, (0.5,), SEED + 20 + lg, dev, **cfg)
            rows.append({"config": f"sizes_{scheme}_lf{lf}", "log2n": lg, **r})
            torch.cuda.empty_cache()
    print(json.dumps({"metric": "size sweep: build/find Gkeys/s against keys per table", "workload": "sizes",
                      "rows": rows}), flush=True)


def run_success(args, world, rank, local):
    """Success rate (Sec. VII-C): the same keys built with 200 different hash
    constant sets per (scheme, load factor); the highest load factor still
    building in >= 99 % of runs. One attempt per build (no retry)."""
    import torch

    import paper_2108_07232_gb300 as G
    import workloads as W
    from paper_2108_07232_gb300 import build as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    n = 1 << 20
    runs = 200
    keys, vals = W.make_keys(n, SEED + 20, device=dev), W.make_values(n, SEED + 20, device=dev)
    grid = {
        "bcht": ({}, (0.95, 0.96, 0.97, 0.98, 0.99)),
        "iht_b32": ({"bucket_size": 32}, (0.88, 0.89, 0.90, 0.91, 0.92, 0.93)),
        "p2bht_b32": ({"bucket_size": 32}, (0.88, 0.89, 0.90, 0.91, 0.92, 0.93)),
        "cuckoo1_h4": ({"num_hashes": 4}, (0.85, 0.86, 0.87, 0.88, 0.89, 0.90)),
    }
    res = {}
    for name, (cfg, lfs) in grid.items():
        scheme = name.split("_")[0]
        res[name] = {}
        for lf in lfs:
            ok = 0
            for r in range(runs):
                t = G.HashTable(scheme, n, lf, seed=SEED + 1000 * r + 7, max_attempts=1, **cfg)
                try:
                    t.build(keys, vals)
                    ok += 1
                except G.GhtError:
                    pass
                del t
            res[name][str(lf)] = ok / runs
        passing = [lf for lf in lfs if res[name][str(lf)] >= 0.99]
        res[name]["max_lf_at_99pct"] = max(passing) if passing else None
    print(json.dumps({"metric": "build success rate over 200 hash-constant sets (2^20 keys)",
                      "workload": "success", "paper_max_lf_at_99pct": {"bcht": 0.98, "iht_b32": 0.91,
                                                                        "p2bht_b32": 0.91, "cuckoo1_h4": 0.88},
                      "rates": res}), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batched":
        run_batched(args, world, rank, local)
        return
    if args.workload == "served":
        run_served(args, world, rank, local)
        return
    if args.workload == "sweep":
        run_sweep(args, world, rank, local)
        return
    if args.workload == "success":
        run_success(args, world, rank, local)
        return
    if args.workload == "sizes":
        run_sizes(args, world, rank, local)
        return
    if args.sharded:
        run_sharded(args, world, rank, local)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
