"""Benchmark: level-synchronous reachability of the BEEM-shaped model on GB300.

One step = one whole reachability run (clear the table, insert init, expand
every BFS level with find-or-put per successor, compact frontiers, count
transitions/deadlocks/levels, accumulate the set digest) of the BEEM-shaped
workload: 12 guarded processes with 4-8 local states, 4 shared int32
variables in [0,4), a critical-state mutex, 16-word (64 B) state vectors,
2^26 buckets.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  `value` = states/s over the K timed steps
(device-resident inputs, CUDA events around the steps), `e2e` = the same
metric through the public C-ABI call reach() with host buffers (model upload,
run, result download inside the timed region).  The same line carries, under
"configs", the other workloads measured in the same run: the tiny
interleaving model, the hash-table benchmark's headline fill with default and
autotuned parameters, the 256-model batch against one model per launch, and
the served Poisson stream (p50/p99 latency, aggregate states/s) against each
job alone (skip them with --no-extra-configs).  `--impl reference` times the
CPU oracle on a bounded sample of the same workload instead.
Under torchrun (N > 1) every rank runs its own replica (no data-path
collective); value = all ranks' states / max over ranks of the time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1004_2772_gb300 import synth  # noqa: E402

METRIC = "states/sec & find_or_put ops/sec on 1 GB300; fraction of HBM random-sector roofline"
# BEEM-shaped: 12 guarded processes, 4 shared vars in [0,4), mutex, W = 16
WORKLOADS = {
    "beem": (dict(seed=22, update_pct=40), 26),
    "beem-medium": (dict(seed=7, update_pct=40), 24),
    "tiny": (None, 18),
    # not reachability of one model: see run_hashtable / run_batch / run_serve
    "hashtable": (None, 26),
    "hashtable-sweep": (None, 0),
    "batch": (None, 0),
    "serve": (None, 0),
    "probe-sweep": (None, 0),
    "part": (dict(seed=22, update_pct=40), 26),
}
LOG2_BUCKETS = 26
MAX_LEVELS = 1 << 14
# DRAM traffic of a kernel (dram__bytes_read.sum + dram__bytes_write.sum, ncu,
# one launch) per unit of work, recorded with the hash of the CUDA sources the
# kernel is compiled from (KERNEL_SOURCES).  A line reports it, scaled to the
# run's units, only while those sources still hash the same and only for the
# workload it was captured on (traffic per unit depends on how much of the table
# L2 holds, so it does not carry over to other sizes); otherwise traffic is null
# and traffic_source says why.  Key: "kernel:workload".
RECORDED_TRAFFIC: dict = {
    "k_reach_persistent:beem-medium": {
        "unit": "transition", "bytes_per_unit": (1311261696 + 766346240) / 21937569,
        "sources_sha": "6e3cc68f02871ba7",
        "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum, "
                   "one launch of the BEEM-shaped medium model (seed 7: 5,478,076 states, 21,937,569 "
                   "transitions, 2^24 buckets): 1.311 GB read + 0.766 GB written"},
    "k_find_or_put_stream:24-0.5-uniform": {
        "unit": "find_or_put", "bytes_per_unit": (1821027584 + 860057088) / 16777216,
        "sources_sha": "7b707ec6b608f7da",
        "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum, "
                   "one fill of a 2^24-bucket table at load 0.5 (16,777,216 calls, 8,388,608 distinct "
                   "16-word keys, uniform): 1.821 GB read + 0.860 GB written"},
    "k_reach_batch:batch64": {
        "unit": "find_or_put", "bytes_per_unit": (11405196288 + 2136117504) / 122061882,
        "sources_sha": "adcbaaa4fff23679",
        "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum, "
                   "one launch of the first 64 models of the batched workload (7,796,054 states, "
                   "122,061,882 find-or-puts): 11.405 GB read + 2.136 GB written"},
}

# the CUDA sources (paper_1004_2772_gb300/csrc) each measured kernel is compiled from
KERNEL_SOURCES = {
    "k_reach_persistent": ["common.cuh", "divide.h", "table.cuh", "coop.cuh", "expand.cuh",
                           "reach_kernels.cuh", "reach.cu", "reach_k16.cu", "reach_k32_lo.cu",
                           "reach_k32_hi.cu", "reach_group.cu"],
    "k_find_or_put_stream": ["common.cuh", "divide.h", "table.cuh", "coop.cuh", "stream.cu"],
    "k_find_or_put": ["common.cuh", "divide.h", "table.cuh", "coop.cuh", "store.cu"],
    "k_reach_batch": ["common.cuh", "divide.h", "table.cuh", "coop.cuh", "expand.cuh", "batch.h",
                      "batch.cu"],
}


def kernel_sources_sha(kernel: str) -> str:
    """sha256 (first 16 hex digits) of the CUDA sources of `kernel`."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1004_2772_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(key: str, units: float):
    """(traffic bytes for `units` units of work or None, a note on its source)."""
    kernel = key.split(":")[0]
    sha = kernel_sources_sha(kernel)
    rec = RECORDED_TRAFFIC.get(key)
    if rec is None:
        note = {"kernel_sources_sha": sha,
                "note": "no DRAM capture recorded for this kernel on this workload"}
        other = {k: v for k, v in RECORDED_TRAFFIC.items() if k.split(":")[0] == kernel}
        if other:  # the same kernel captured on a smaller workload, for reference
            note["smaller_workload_captures"] = {k: {"bytes_per_unit": v["bytes_per_unit"], "unit": v["unit"],
                                                     "current": v["sources_sha"] == sha}
                                                 for k, v in other.items()}
        return None, note
    if rec["sources_sha"] != sha:
        return None, {"kernel_sources_sha": sha, "capture_sources_sha": rec["sources_sha"],
                      "note": "the kernel sources changed since the DRAM capture"}
    return rec["bytes_per_unit"] * units, {"kernel_sources_sha": sha, "unit": rec["unit"],
                                           "bytes_per_unit": rec["bytes_per_unit"],
                                           "capture": rec["capture"]}


def workload_model(name="beem"):
    spec, _ = WORKLOADS[name]
    if spec is None:
        return synth.tiny_interleaving_model()
    return synth.beem_shaped_model(**spec)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "clocks.mem,temperature.gpu,pci.bus_id")

    def __init__(self, gpu_index: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        self.gpu = ids[gpu_index] if gpu_index < len(ids) else str(gpu_index)
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        extra = {"power_w": [], "mem_mhz": [], "temp_c": []}
        bus = None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
            for key, i in (("power_w", 3), ("mem_mhz", 9), ("temp_c", 10)):
                try:
                    extra[key].append(float(parts[i]))
                except (ValueError, IndexError):
                    pass
            if len(parts) > 11:
                bus = parts[11]
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        out = {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
               "samples": len(sm)}
        for key, vals in extra.items():  # medians, for comparing runs across boxes
            if vals:
                out[key] = sorted(vals)[len(vals) // 2]
        if bus:
            out["pci_bus_id"] = bus
        return out


def algorithmic_bytes(states, transitions, state_words=16):
    """Minimum HBM bytes of one run (per-unit figures):
    expanded state: data row read (16*ceil(W/4) B) + 4 B frontier read;
    duplicate find-or-put: one 32 B bucket sector + the data row compared;
    new find-or-put: one 32 B bucket sector read + written back, data row
    written, 4 B frontier write."""
    row = 16 * ((state_words + 3) // 4)
    new = states - 1
    dup = transitions - new
    return states * (row + 4) + dup * (32 + row) + new * (64 + row + 4)


def random_bound_s(states, transitions, rates, hbm_gbs, state_words=16):
    """Seconds one run would take if every random access ran at the
    probe-measured random-access rate of this GPU (`vss_probe_random`) and the
    frontier rows streamed at copy bandwidth:
      per transition        one random 32 B bucket-sector read
      per duplicate         one random row read (the compare): a 32 B read for
                            rows of 32 B, else row/64 random 64 B reads
      per new state         row/32 + 1 random 32 B sector writes (row + bucket write-back)
      per expanded state    its frontier row read and, once, written (streamed)."""
    row = 16 * ((state_words + 3) // 4)
    new = states - 1
    dup = transitions - new
    row_read = 1.0 / rates[0] if row <= 32 else (row / 64) / rates[1]
    return (transitions / rates[0] + dup * row_read + (row // 32 + 1) * new / rates[2]
            + 2 * states * row / (hbm_gbs * 1e9))


def random_roofline(states, transitions, kernel_ms, rates, hbm_gbs, state_words=16):
    """The run's time at the random-access bound (random_bound_s) against the
    measured kernel time."""
    t = random_bound_s(states, transitions, rates, hbm_gbs, state_words)
    return {"bound_ms": t * 1e3, "kernel_ms": kernel_ms, "frac": (t * 1e3) / kernel_ms,
            "find_or_put_bound_per_s": transitions / t,
            "probe_rates_per_s": {"read32": rates[0], "read64": rates[1], "write32": rates[2],
                                  "atomic32": rates[3]},
            "unit": "fraction of the random-access bound (probe-measured rates)"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_baseline(model):
    """The oracle, as it stands, on a bounded sample: BFS truncated after a
    fixed number of stored states (about 10 s on one Grace core)."""
    import oracle
    sample = 6_000_000
    t = time.perf_counter()
    r = oracle.reach(model, max_states=sample)
    dt = time.perf_counter() - t
    return {"value": r.states / dt, "unit": "states/s", "cores": 1, "kind": "oracle",
            "sample": f"first {r.states} states (BFS truncated) of {model.name}, "
                      f"single-threaded std::unordered_set BFS, {dt:.1f} s"}


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle, timed on the host, rank 0 only."""
    if rank != 0:
        return
    import oracle
    model = workload_model(args.workload)
    sample = int(os.environ.get("BENCH_REF_SAMPLE", "1000000"))
    for _ in range(args.warmup):
        oracle.reach(model, max_states=sample // 4)
    t0 = time.perf_counter()
    states = 0
    for _ in range(args.steps):
        r = oracle.reach(model, max_states=sample)
        states += r.states
    dt = time.perf_counter() - t0
    v = states / dt
    line = {"metric": METRIC, "value": v, "unit": "states/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": model.name, "sample_states": sample, "log2_buckets": LOG2_BUCKETS},
            "cpu_baseline": {"value": v, "unit": "states/s", "cores": 1, "kind": "oracle",
                             "sample": f"BFS truncated at {sample} states per step"},
            "e2e": {"value": v, "unit": "states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="persistent", choices=["persistent", "per-level", "graph"])
    ap.add_argument("--line-buckets", type=int, default=32)
    ap.add_argument("--group-lanes", type=int, default=1,
                    help="lanes per successor in the reachability kernel (2, 4, 8: cooperative "
                         "probing of lines of 4G buckets; the line length follows)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the tiny / hash-table / batch / served measurements of the default line")
    ap.add_argument("--workload", default="beem", choices=sorted(WORKLOADS))
    ap.add_argument("--log2-buckets", type=int, default=0, help="0 = the workload's size")
    ap.add_argument("--load-factor", type=float, default=0.75, help="hashtable: keys / buckets")
    ap.add_argument("--dist", default="uniform", choices=["uniform", "zipf"], help="hashtable reuse")
    ap.add_argument("--key-mode", default="fused", choices=["fused", "api"],
                    help="hashtable: keys generated in registers, or materialised batches")
    ap.add_argument("--autotune", action="store_true", help="hashtable: tune parameters first")
    ap.add_argument("--duration", type=float, default=10.0, help="serve: seconds of arrivals")
    ap.add_argument("--models", type=int, default=256, help="batch: number of models")
    ap.add_argument("--probe-gib", type=float, default=16.0, help="buffer size (GiB) of the random-access probe every workload runs for its roofline")
    ap.add_argument("--probe-modes", default="0,1,2,3,4,5,6,7,8,9,10,11,12", help="probe-sweep: modes")
    ap.add_argument("--probe-default-shape", action="store_true",
                    help="probe-sweep: only the default shape (8 in flight, 8 blocks/SM, 256 threads)")
    ap.add_argument("--probe-reps", type=int, default=3, help="probe-sweep: timed runs per shape")
    ap.add_argument("--parts", type=int, default=4, help="part: owner partitions")
    ap.add_argument("--exchange-rows", type=int, default=1 << 23,
                    help="part: rows of one exchange chunk (outbox and inbox each)")
    args = ap.parse_args()
    global LOG2_BUCKETS
    LOG2_BUCKETS = args.log2_buckets or WORKLOADS[args.workload][1]
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_1004_2772_gb300 import _build, binding
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    binding.load()
    if args.workload in ("hashtable", "hashtable-sweep", "batch", "serve", "probe-sweep", "part"):
        {"hashtable": run_hashtable, "hashtable-sweep": run_hashtable_sweep, "batch": run_batch,
         "serve": run_serve, "probe-sweep": run_probe_sweep,
         "part": run_part}[args.workload](args, world, rank, local, dev)
        return

    model = workload_model(args.workload)
    mode = {"persistent": binding.REACH_PERSISTENT, "per-level": binding.REACH_PER_LEVEL,
            "graph": binding.REACH_GRAPH}[args.mode]
    # the context is allocated first, as in a process that only runs
    # reachability: a probe buffer of many GB allocated and freed before it
    # moves the context elsewhere in device memory, and the kernel's time
    # with it (by several per cent either way)
    group = {} if args.group_lanes == 1 else {"group_lanes": args.group_lanes}
    line_buckets = args.line_buckets if args.group_lanes == 1 else 4 * args.group_lanes
    ctx = binding.ReachContext(LOG2_BUCKETS, model.state_words, max_levels=MAX_LEVELS,
                               line_buckets=line_buckets, **group)
    ctx.load(model)
    stream = torch.cuda.current_stream()
    # random-access rates of this GPU (the random-sector roofline's denominators):
    # each mode's plateau over the probe shapes
    rates = binding.random_access_rates(gib=args.probe_gib, n_access=1 << 28)

    # warm-up (also yields the result that every timed step must reproduce)
    for _ in range(max(3, args.warmup)):
        ctx.run(mode)
        ref = ctx.result()

    # timed: device-resident inputs, K steps bracketed by barrier + sync
    kernel_ms, launches = 0.0, 0
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.run(mode)
        e1.record(stream)
        torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / args.steps
    # the dominant kernel's device time: the mean over the timed launches, from
    # the CUDA events the library records around each launch on its stream
    if mode == binding.REACH_PERSISTENT:
        times = ctx.run_times(min(args.steps, 64))
        kernel_ms = float(np.mean(times))
    else:
        kernel_ms = ctx.last_timing()[0]
    launches = ctx.last_timing()[1]
    got = ctx.result()
    assert (got.states, got.transitions, got.digest, got.level_sizes) == (
        ref.states, ref.transitions, ref.digest, ref.level_sizes), "timed runs disagree"
    barrier(world)
    t_max = max_over_ranks(step_ms, world, dev)
    states_all = sum_over_ranks(float(got.states), world, dev)
    trans_all = sum_over_ranks(float(got.transitions), world, dev)
    value = states_all / (t_max / 1000.0)

    # end to end: the public call with host buffers (model upload, run, result download)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = ctx.reach(model, mode=mode)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1000 / args.steps
    assert r.states == ref.states and r.digest == ref.digest
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    h2d = model.nbytes()
    d2h = 64 + 64 + 8 * len(r.level_sizes)
    ctx.close()
    del ctx
    torch.cuda.empty_cache()

    peak, which = peaks()
    tab_bytes = binding.ht_bytes(LOG2_BUCKETS, model.state_words)
    if tab_bytes > 129e6:
        l2_note = (f"inputs larger than L2 ({tab_bytes / 1e9:.1f} GB table per step; bucket array "
                   f"{(4 << LOG2_BUCKETS) >> 20} MiB)")
    else:
        l2_note = (f"L2-resident working set ({tab_bytes / 1e6:.0f} MB table), not flushed between "
                   "steps: a latency-bound configuration")
    alg = algorithmic_bytes(got.states, got.transitions, model.state_words)
    achieved = alg / (kernel_ms / 1000.0) / 1e9
    kname = {0: "k_reach_persistent", 1: "k_reach_level", 2: "k_reach_step"}[mode]
    traffic, traffic_src = (recorded_traffic(f"{kname}:{args.workload}", got.transitions)
                            if args.group_lanes == 1 and line_buckets == 32 else
                            (None, {"note": "DRAM captures are recorded for the default line layout only"}))
    line = {
        "metric": METRIC, "value": value, "unit": "states/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": model.name, "states": got.states, "transitions": got.transitions,
                   "levels": len(got.level_sizes), "state_words": model.state_words,
                   "log2_buckets": LOG2_BUCKETS, "line_buckets": line_buckets,
                   "group_lanes": args.group_lanes,
                   "mode": args.mode, "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": l2_note},
        "find_or_put_ops_per_s": trans_all / (t_max / 1000.0),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                     "kernel": kname, "kernel_ms": kernel_ms, "algorithmic_bytes": alg,
                     "peak_source": which},
        "random_roofline": random_roofline(got.states, got.transitions, kernel_ms, rates, peak,
                                           model.state_words),
        "e2e": {"value": states_all / (e2e_ms / 1000.0), "unit": "states/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches * args.steps,
        "clocks": clocks.summary(),
    }
    if not args.no_extra_configs and args.workload == "beem" and mode == binding.REACH_PERSISTENT:
        line["configs"] = extra_configs(args, world, local, dev, rates)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(model)
        line["cpu_baseline"]["host_cores_available"] = os.cpu_count()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def base_line(args, world, metric, value, unit, ms_per_step, config, higher=True):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": higher,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config}


def probe_rates_dict(rates):
    return {"read32": rates[0], "read64": rates[1], "write32": rates[2], "atomic32": rates[3]}


# ---------------------------------------------------------------------------
# The other workloads, as functions returning a result dict (used both by
# their own --workload lines and by the default line's "configs").
# ---------------------------------------------------------------------------

def tiny_stats(steps, local):
    """The tiny interleaving model (10^5 states, 2^18 buckets, L2-resident):
    the three level drivers; value = states/s of the persistent driver."""
    import torch
    from paper_1004_2772_gb300 import binding
    m = synth.tiny_interleaving_model()
    ctx = binding.ReachContext(18, m.state_words, max_levels=MAX_LEVELS)
    ctx.load(m)
    out = {"workload": m.name, "unit": "states/s"}
    with ClockSampler(local) as clocks:
        for name, mode in (("persistent", binding.REACH_PERSISTENT), ("graph", binding.REACH_GRAPH),
                           ("per_level", binding.REACH_PER_LEVEL)):
            for _ in range(3):
                ctx.run(mode)
            ref = ctx.result()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                ctx.run(mode)
            e1.record()
            torch.cuda.synchronize()
            got = ctx.result()
            assert (got.states, got.digest, got.level_sizes) == (ref.states, ref.digest, ref.level_sizes)
            out[f"{name}_ms_per_run"] = e0.elapsed_time(e1) / steps
    ctx.close()
    out["value"] = got.states / (out["persistent_ms_per_run"] / 1e3)
    out["states"], out["levels"] = got.states, len(got.level_sizes)
    out["l2"] = "L2-resident (6 MB table), not flushed: latency-bound"
    out["clocks"] = clocks.summary()
    return out


def hashtable_point(log2, lf, dist, key_mode, params, steps, warmup, rates, local):
    """One fill of a 2^log2 table to load factor lf per step (2 * lf * 2^log2
    find-or-put calls, half of them repeating an earlier key uniformly or by
    Zipf(1.1)); value = find-or-put calls per second."""
    import torch
    from paper_1004_2772_gb300 import binding
    n_ids = int(lf * (1 << log2))
    calls = 2 * n_ids
    zipf = synth.zipf_table(n_ids) if dist == "zipf" else None
    tab = binding.Table(log2, 16, **params)
    tab_gb = binding.ht_bytes(log2, 16) / 1e9
    keys = tab.gen_keys(1, n_ids, 0, calls, zipf) if key_mode == "api" else None

    def step():
        tab.clear()
        if keys is None:
            return tab.find_or_put_stream(1, n_ids, 0, calls, zipf, sync=False)
        return tab.find_or_put(keys, want_idx=True)
    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the last fill must have stored exactly the fill's distinct keys
    st = tab.stats()
    assert st.stored == n_ids and st.error == 0, (st.stored, n_ids)
    tab.close()
    del keys
    torch.cuda.empty_cache()
    dup, new = calls - n_ids, n_ids
    alg = calls * 32 + dup * 64 + new * (64 + 32) + (calls * (64 + 5) if key_mode == "api" else 0)
    bound_s = hashtable_bound_s(calls, n_ids, rates, key_mode == "api")
    peak, which = peaks()
    kname = "k_find_or_put_stream" if key_mode == "fused" else "k_find_or_put"
    traffic, src = (recorded_traffic(f"{kname}:{log2}-{lf}-{dist}", calls) if not params
                    else (None, {"note": "no DRAM capture recorded for these parameters"}))
    return {"workload": f"hashtable-W16-2^{log2}-lf{lf}-{dist}-{key_mode}", "value": calls / (ms / 1e3),
            "unit": "find_or_put/s", "ms_per_fill": ms, "calls_per_fill": calls, "distinct_keys": n_ids,
            "params": params, "steps": steps,
            "l2": f"inputs larger than L2 (table {tab_gb:.1f} GB)",
            "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": traffic, "traffic_source": src,
                         "kernel": kname, "algorithmic_bytes": alg, "peak_source": which},
            "random_roofline": {"bound_ms": bound_s * 1e3, "frac": bound_s * 1e3 / ms,
                                "probe_rates_per_s": probe_rates_dict(rates)},
            "gpu_launches": steps * (1 if key_mode == "fused" else 1),
            "clocks": clocks.summary()}


def run_hashtable(args, world, rank, local, dev):
    """Hash-table benchmark: one step = one fill (hashtable_point)."""
    from paper_1004_2772_gb300 import autotune, binding
    params = {"line_buckets": args.line_buckets} if args.line_buckets != 32 else {}
    tuned = None
    if args.autotune:
        tuned = autotune.tune_table(LOG2_BUCKETS, args.load_factor, args.dist, cache_path=None)
        params = dict(tuned["best"])
    rates = binding.random_access_rates(gib=args.probe_gib, n_access=1 << 28)
    r = hashtable_point(LOG2_BUCKETS, args.load_factor, args.dist, args.key_mode, params, args.steps,
                        args.warmup, rates, local)
    t_max = max_over_ranks(r["ms_per_fill"], world, dev)
    ops = sum_over_ranks(float(r["calls_per_fill"]), world, dev) / (t_max / 1e3)
    line = base_line(args, world, "find_or_put ops/sec on 1 GB300 (hash-table benchmark)", ops,
                     "find_or_put/s", t_max,
                     {"workload": r["workload"], "calls_per_step": r["calls_per_fill"],
                      "distinct_keys": r["distinct_keys"], "params": params, "l2": r["l2"]})
    for k in ("roofline", "random_roofline", "gpu_launches", "clocks"):
        line[k] = r[k]
    if tuned:
        line["autotune"] = {"best": tuned["best"], "candidates": len(tuned["all"])}
    if rank == 0:
        print(json.dumps(line), flush=True)


def hashtable_bound_s(calls, n_ids, rates, api):
    """Seconds the fill would take at the probe-measured random-access rates:
    a 32 B sector read per call, a 64 B row read per repeat, a sector CAS plus
    a 64 B row write per new key (streamed keys and outputs at copy speed)."""
    dup, new = calls - n_ids, n_ids
    t = calls / rates[0] + dup / rates[1] + 3 * new / rates[2]
    if api:
        t += calls * (64 + 5) / (peaks()[0] * 1e9)
    return t


def run_hashtable_sweep(args, world, rank, local, dev):
    """The hash-table benchmark grid: 2^n buckets for n in 24..28, load factors
    0.5 / 0.75 / 0.9, uniform and Zipf(1.1) reuse, keys in registers (fused)
    and materialised (batch API); at least 10^9 timed calls per point (whole
    fills repeated).  value = calls/s at 2^26, LF 0.75, uniform, fused."""
    import torch
    from paper_1004_2772_gb300 import binding, synth
    rates = binding.random_access_rates(gib=args.probe_gib, n_access=1 << 28)
    min_calls = int(float(os.environ.get("BENCH_SWEEP_MIN_CALLS", "1e9")))
    points = []
    t_all = time.perf_counter()
    with ClockSampler(local) as clocks:
        for log2 in (24, 25, 26, 27, 28):
            for lf in (0.5, 0.75, 0.9):
                n_ids = int(lf * (1 << log2))
                calls = 2 * n_ids
                fills = max(1, -(-min_calls // calls))
                tab = binding.Table(log2, 16)
                for dist in ("uniform", "zipf"):
                    zipf = synth.zipf_table(n_ids) if dist == "zipf" else None
                    for mode in ("fused", "api"):
                        keys = tab.gen_keys(1, n_ids, 0, calls, zipf) if mode == "api" else None

                        def fill():
                            tab.clear()
                            if keys is None:
                                tab.find_or_put_stream(1, n_ids, 0, calls, zipf, sync=False)
                            else:
                                tab.find_or_put(keys, want_idx=True)
                        fill()
                        torch.cuda.synchronize()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        for _ in range(fills):
                            fill()
                        e1.record()
                        torch.cuda.synchronize()
                        ms = e0.elapsed_time(e1) / fills
                        st = tab.stats()
                        assert st.stored == n_ids and st.error == 0, (log2, lf, dist, mode)
                        bound = hashtable_bound_s(calls, n_ids, rates, keys is not None)
                        points.append({"log2_buckets": log2, "load_factor": lf, "dist": dist,
                                       "keys": mode, "ops_per_s": calls / (ms / 1e3),
                                       "ms_per_fill": ms, "timed_calls": calls * fills,
                                       "random_roofline_frac": bound * 1e3 / ms})
                        del keys
                tab.close()
                torch.cuda.empty_cache()
    head = [p for p in points if p["log2_buckets"] == 26 and p["load_factor"] == 0.75
            and p["dist"] == "uniform" and p["keys"] == "fused"][0]
    line = base_line(args, world, "find_or_put ops/sec on 1 GB300 (hash-table benchmark sweep)",
                     head["ops_per_s"], "find_or_put/s", head["ms_per_fill"],
                     {"workload": "hashtable-sweep-W16-2^24..2^28-lf0.5,0.75,0.9-uniform,zipf-fused,api",
                      "l2": "tables 1.1-18 GB, larger than L2", "min_timed_calls_per_point": min_calls})
    line["points"] = points
    line["sweep_seconds"] = time.perf_counter() - t_all
    line["probe_rates_per_s"] = {"read32": rates[0], "read64": rates[1], "write32": rates[2],
                                 "atomic32": rates[3]}
    line["gpu_launches"] = sum(-(-min_calls // (2 * int(p["load_factor"] * (1 << p["log2_buckets"]))))
                               for p in points)
    line["clocks"] = clocks.summary()
    if rank == 0:
        print(json.dumps(line), flush=True)


def batch_stats(models, steps, warmup, rates, local):
    """The batched models in one persistent launch replayed as a CUDA graph
    (value = states/s), against one model per launch through reach() (each
    model alone, on a context sized for it)."""
    import torch
    from paper_1004_2772_gb300 import binding
    bt = binding.ReachBatch(models, max_levels=4096)
    for _ in range(max(3, warmup)):
        bt.run(use_graph=True)
    ref, grows, st = bt.results()
    assert st == 0
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            bt.run(use_graph=True)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    got, grows, st = bt.results()
    assert st == 0 and [r.digest for r in got] == [r.digest for r in ref]
    bt.close()
    del bt
    torch.cuda.empty_cache()
    states = sum(r.states for r in got)
    # one model per launch (the plain path), contexts sized per model; device
    # time of each run from the library's events, and the host wall time
    ctxs, dev_ms, t0 = {}, 0.0, time.perf_counter()
    for m in models:
        lg = max(10, int(np.ceil(np.log2(float(np.prod(m.n_local)) / 0.5))))
        ctxs.setdefault(lg, binding.ReachContext(lg, 32, max_levels=4096))
        r = ctxs[lg].reach(m)
        assert r.status == 0
        dev_ms += ctxs[lg].last_timing()[0]
    torch.cuda.synchronize()
    loop_ms = (time.perf_counter() - t0) * 1e3
    for c in ctxs.values():
        c.close()
    del ctxs
    torch.cuda.empty_cache()
    peak, which = peaks()
    alg = sum(algorithmic_bytes(r.states, r.transitions, m.state_words) for m, r in zip(models, got))
    bound_s = sum(random_bound_s(r.states, r.transitions, rates, peak, m.state_words)
                  for m, r in zip(models, got))
    fops = sum(r.transitions for r in got)
    traffic, src = recorded_traffic(f"k_reach_batch:batch{len(models)}", fops)
    return {"workload": f"batched-{len(models)}-interleaving-models", "value": states / (ms / 1e3),
            "unit": "states/s", "ms_per_batch": ms, "models": len(models), "states": states,
            "table_grows": int(sum(grows)), "graph": True, "steps": steps,
            "l2": "inputs larger than L2 (tables and frontiers, GBs)",
            "find_or_put_ops_per_s": fops / (ms / 1e3),
            "one_model_per_launch": {"wall_ms": loop_ms, "device_ms": dev_ms,
                                     "states_per_s": states / (loop_ms / 1e3),
                                     "batch_speedup_vs_wall": loop_ms / ms},
            "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": traffic, "traffic_source": src,
                         "kernel": "k_reach_batch", "algorithmic_bytes": alg, "peak_source": which},
            "random_roofline": {"bound_ms": bound_s * 1e3, "kernel_ms": ms, "frac": bound_s * 1e3 / ms,
                                "probe_rates_per_s": probe_rates_dict(rates),
                                "unit": "fraction of the random-access bound (probe-measured rates)"},
            "gpu_launches": steps, "clocks": clocks.summary()}


def run_batch(args, world, rank, local, dev):
    """Batched reachability: one step = the 256 seeded interleaving models of
    uneven size (3-12 processes, 8-32 words, 10^3-10^6 states) in one
    persistent launch replayed as a CUDA graph; compared with one model per
    launch."""
    from paper_1004_2772_gb300 import binding
    models = synth.batched_models(count=args.models, first_seed=1)
    rates = binding.random_access_rates(gib=args.probe_gib, n_access=1 << 28)
    r = batch_stats(models, args.steps, args.warmup, rates, local)
    t_max = max_over_ranks(r["ms_per_batch"], world, dev)
    value = sum_over_ranks(float(r["states"]), world, dev) / (t_max / 1e3)
    line = base_line(args, world, f"states/sec on 1 GB300 (batched reachability, {len(models)} models)",
                     value, "states/s", t_max,
                     {"workload": r["workload"], "models": r["models"], "states": r["states"],
                      "table_grows": r["table_grows"], "graph": True, "l2": r["l2"]})
    for k in ("one_model_per_launch", "find_or_put_ops_per_s", "roofline", "random_roofline",
              "gpu_launches", "clocks"):
        line[k] = r[k]
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_stats(jobs, slots_list, plain, local):
    """The served stream submitted in real time (arrival times of `jobs`) to a
    server of each slot count (HBM budget = 85% of free memory): aggregate
    states/s, p50/p99 latency; with `plain`, each job alone through reach()
    in arrival order (device time of each run, host overheads excluded)."""
    import gc

    import torch
    from paper_1004_2772_gb300 import binding
    gc.collect()
    torch.cuda.empty_cache()  # earlier measurements' memory back to the driver before sizing
    free, _ = torch.cuda.mem_get_info()
    out = {}
    with ClockSampler(local) as clocks:
        for slots in slots_list:
            srv = binding.Server(budget_bytes=int(free * 0.85), n_slots=slots, max_levels=4096)
            srv.submit(jobs[0][1])
            while not srv.poll(want_levels=False):
                time.sleep(0.001)
            done, k, t0 = [], 0, time.perf_counter()
            while len(done) < len(jobs):
                now = time.perf_counter() - t0
                while k < len(jobs) and jobs[k][0] <= now:
                    srv.submit(jobs[k][1])
                    k += 1
                done += srv.poll(want_levels=False)
                time.sleep(0.0001)  # the client polls completions every 0.1 ms
            span = time.perf_counter() - t0
            lat = np.array([d.latency_s for d in done]) * 1e3
            queue = np.array([d.admit_s - d.submit_s for d in done]) * 1e3
            run = np.array([d.done_s - d.admit_s for d in done]) * 1e3
            size = np.array([d.result.states for d in done], dtype=np.float64)
            assert all(d.result.status == 0 for d in done)
            by_size = {}
            for lo, hi in ((1e4, 1e5), (1e5, 1e6), (1e6, 1e7), (1e7, 1e9)):
                sel = (size >= lo) & (size < hi)
                if sel.any():
                    by_size[f"{lo:.0e}-{hi:.0e}"] = {"jobs": int(sel.sum()),
                                                      "p50_ms": float(np.percentile(lat[sel], 50))}
            out[slots] = {"span_s": span, "states": int(size.sum()),
                          "states_per_s": float(size.sum()) / span,
                          "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                          "max_ms": float(lat.max()), "kernel_launches": srv.status()["kernel_launches"],
                          "queue_p50_ms": float(np.percentile(queue, 50)),
                          "run_p50_ms": float(np.percentile(run, 50)), "p50_ms_by_states": by_size}
            srv.close()
            del srv
            torch.cuda.empty_cache()
    if plain:
        # the plain path: each job alone through reach() on a context sized for
        # it, in arrival order (a job starts when it has arrived and the
        # previous one finished)
        ctxs, t_free, lat_plain = {}, 0.0, []
        for arrival, m in jobs:
            bound = float(np.prod(np.asarray(m.n_local, dtype=np.float64)))
            lg = max(10, int(np.ceil(np.log2(bound / 0.5))))
            ctx = ctxs.get(lg) or binding.ReachContext(lg, m.state_words, max_levels=4096)
            r = ctx.reach(m)
            assert r.status == 0
            run_s = ctx.last_timing()[0] / 1e3
            start = max(arrival, t_free)
            t_free = start + run_s
            lat_plain.append((t_free - arrival) * 1e3)
            if lg <= 24:
                ctxs[lg] = ctx
            else:
                ctx.close()
                del ctx
                torch.cuda.empty_cache()
        for ctx in ctxs.values():
            ctx.close()
        del ctxs
        torch.cuda.empty_cache()
        lat_plain = np.array(lat_plain)
        out["plain"] = {"p50_ms": float(np.percentile(lat_plain, 50)),
                        "p99_ms": float(np.percentile(lat_plain, 99)),
                        "note": "device time of each job alone via reach(), queued in arrival order; "
                                "host overheads excluded"}
    out["clocks"] = clocks.summary()
    return out


def run_serve(args, world, rank, local, dev):
    """Served reachability: a Poisson stream (20 jobs/s) of interleaving jobs of
    log-uniform size 10^4..2*10^8 states (W = 16) submitted in real time to the
    server (a job that finds the GPU idle runs on the single-model kernel,
    queues go to the continuous-batching kernel); reports aggregate states/s
    and p50/p99 latency, the same stream with one slot, and each job alone
    through reach() in arrival order."""
    jobs = synth.served_jobs(seed=5, rate=20.0, duration_s=args.duration)
    out = serve_stats(jobs, (64, 1), True, local)
    c = out[64]
    line = base_line(args, world, "states/sec on 1 GB300 (served reachability, Poisson 20 jobs/s)",
                     c["states_per_s"], "states/s", c["span_s"] * 1e3 / max(1, len(jobs)),
                     {"workload": f"served-poisson20-{len(jobs)}jobs-1e4..2e8-W16", "slots": 64,
                      "jobs": len(jobs)})
    line["latency_ms"] = {"p50": c["p50_ms"], "p99": c["p99_ms"], "max": c["max_ms"],
                          "queue_p50": c["queue_p50_ms"], "run_p50": c["run_p50_ms"],
                          "p50_by_states": c["p50_ms_by_states"]}
    o = out[1]
    line["one_job_at_a_time"] = {"p50_ms": o["p50_ms"], "p99_ms": o["p99_ms"],
                                 "queue_p50_ms": o["queue_p50_ms"], "run_p50_ms": o["run_p50_ms"],
                                 "p50_by_states": o["p50_ms_by_states"], "states_per_s": o["states_per_s"]}
    line["plain_reach_in_arrival_order"] = out["plain"]
    line["gpu_launches"] = c["kernel_launches"]
    line["clocks"] = out["clocks"]
    if rank == 0:
        print(json.dumps(line), flush=True)


def extra_configs(args, world, local, dev, rates):
    """The default line's other workloads (one GPU each, rank 0's numbers)."""
    from paper_1004_2772_gb300 import autotune
    out = {"tiny": tiny_stats(max(10, args.steps), local)}
    steps = max(5, min(args.steps, 20))
    out["hashtable"] = hashtable_point(26, 0.75, "uniform", "fused", {}, steps, args.warmup, rates, local)
    t0 = time.perf_counter()
    tuned = autotune.tune_table(26, 0.75, "uniform", cache_path=None)
    tune_s = time.perf_counter() - t0
    ht = hashtable_point(26, 0.75, "uniform", "fused", dict(tuned["best"]), steps, args.warmup, rates,
                         local)
    ht["autotune"] = {"best": tuned["best"], "candidates": len(tuned["all"]), "seconds": tune_s}
    out["hashtable_autotuned"] = ht
    out["batch"] = batch_stats(synth.batched_models(count=256, first_seed=1), max(3, min(args.steps, 10)),
                               args.warmup, rates, local)
    jobs = synth.served_jobs(seed=5, rate=20.0, duration_s=10.0)
    sv = serve_stats(jobs, (64,), True, local)
    c = sv[64]
    out["serve"] = {"workload": f"served-poisson20-{len(jobs)}jobs-1e4..2e8-W16", "value": c["states_per_s"],
                    "unit": "states/s", "slots": 64, "jobs": len(jobs), "span_s": c["span_s"],
                    "latency_ms": {"p50": c["p50_ms"], "p99": c["p99_ms"], "max": c["max_ms"],
                                   "queue_p50": c["queue_p50_ms"], "run_p50": c["run_p50_ms"],
                                   "p50_by_states": c["p50_ms_by_states"]},
                    "plain_reach_in_arrival_order": sv["plain"], "gpu_launches": c["kernel_launches"],
                    "clocks": sv["clocks"]}
    return out


def run_probe_sweep(args, world, rank, local, dev):
    """The random-access probe in every swept shape (accesses in flight per
    thread x blocks per SM x threads per block) for every mode, over a 16 GiB
    buffer: the plateau of each mode is the roofline denominator bench.py
    uses.  value = the plateau of 32-byte sector reads."""
    from paper_1004_2772_gb300 import binding
    modes = tuple(int(x) for x in args.probe_modes.split(","))
    shapes = {m: [(8, 8, 256)] for m in modes} if args.probe_default_shape else None
    with ClockSampler(local) as clocks:
        rows = binding.probe_sweep(gib=args.probe_gib, n_access=1 << 28, modes=modes,
                                   reps=args.probe_reps, shapes=shapes)
    best = {m: max((r for r in rows if r["mode"] == m), key=lambda r: r["per_s"]) for m in modes}
    line = base_line(args, world, "random 32-byte sector reads/sec on 1 GB300 (probe plateau)",
                     best[modes[0]]["per_s"], "accesses/s", None,
                     {"workload": f"random-access-probe-{args.probe_gib:g}GiB", "accesses_per_run": 1 << 28,
                      "modes": list(modes), "l2": f"{args.probe_gib:g} GiB buffer, larger than L2"})
    line["plateau"] = {binding.PROBE_MODES[m]: best[m] for m in modes}
    line["rows"] = rows
    line["clocks"] = clocks.summary()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_part(args, world, rank, local, dev):
    """The BEEM-shaped workload on K owner partitions of one GPU (static
    partitioning: successors exchanged between owners every level) against
    the shared table (the paper's comparison of the two architectures).
    value = states/s of the partitioned run (host-driven levels; wall time of
    part_reach_run, which synchronises once per level)."""
    import torch
    from paper_1004_2772_gb300 import binding
    model = workload_model("part")
    K = args.parts
    lg = LOG2_BUCKETS - (K.bit_length() - 1)
    pr = binding.PartReach(K, lg, model.state_words, exchange_rows=args.exchange_rows)
    for _ in range(max(1, args.warmup)):
        ref, parts, ex = pr.run(model)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            got, parts, ex = pr.run(model)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / args.steps
    assert (got.states, got.digest, got.level_sizes) == (ref.states, ref.digest, ref.level_sizes)
    pr.close()
    del pr
    torch.cuda.empty_cache()
    ctx = binding.ReachContext(LOG2_BUCKETS, model.state_words, max_levels=MAX_LEVELS)
    ctx.load(model)
    for _ in range(3):
        ctx.run(binding.REACH_PERSISTENT)
    shared = ctx.result()
    for _ in range(args.steps):
        ctx.run(binding.REACH_PERSISTENT)
    shared_ms = float(np.mean(ctx.run_times(min(args.steps, 64))))
    ctx.close()
    assert (shared.states, shared.digest) == (got.states, got.digest)
    line = base_line(args, world, f"states/sec on 1 GB300 (owner-partitioned reachability, {K} owners)",
                     got.states / (ms / 1e3), "states/s", ms,
                     {"workload": model.name, "parts": K, "log2_buckets_per_part": lg,
                      "exchange_rows": args.exchange_rows,
                      "states": got.states, "transitions": got.transitions,
                      "l2": "inputs larger than L2 (tables and frontiers, GBs)"})
    line["exchanged"] = ex
    line["exchanged_frac"] = ex / got.transitions
    line["part_states"] = parts
    line["shared_table"] = {"ms_per_run": shared_ms, "states_per_s": shared.states / (shared_ms / 1e3)}
    line["clocks"] = clocks.summary()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
