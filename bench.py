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
run, result download inside the timed region).  `--impl reference` times the
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1004_2772_gb300 import synth  # noqa: E402

METRIC = "states/sec & find_or_put ops/sec on 1 GB300; fraction of HBM random-sector roofline"
# BEEM-shaped: 12 guarded processes, 4 shared vars in [0,4), mutex, W = 16
WORKLOADS = {
    "beem": (dict(seed=22, update_pct=40), 26),
    "beem-medium": (dict(seed=7, update_pct=40), 24),
    "tiny": (None, 18),
}
LOG2_BUCKETS = 26
MAX_LEVELS = 1 << 14


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
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

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
                 "--format=csv,noheader,nounits", "-lms", "200"],
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


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


def random_roofline(states, transitions, kernel_ms, rates, hbm_gbs, state_words=16):
    """Time the run would take if every random access ran at the probe-measured
    random-access rate of this GPU (`vss_probe_random`) and the frontier rows
    streamed at copy bandwidth:
      per transition        one random 32 B bucket-sector read
      per duplicate         one random 64 B row read (the compare)
      per new state         three random 32 B sector writes (row + bucket write-back)
      per expanded state    its frontier row read and, once, written (streamed)."""
    row = 16 * ((state_words + 3) // 4)
    new = states - 1
    dup = transitions - new
    t = (transitions / rates[0] + dup / rates[1] + 3 * new / rates[2]
         + 2 * states * row / (hbm_gbs * 1e9))
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


def cpu_baseline(model, seconds_target=15.0):
    """The oracle, as it stands, on a bounded sample: BFS truncated after a
    fixed number of stored states."""
    import oracle
    sample = 1_500_000
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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="persistent", choices=["persistent", "per-level"])
    ap.add_argument("--line-buckets", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="beem", choices=sorted(WORKLOADS))
    ap.add_argument("--log2-buckets", type=int, default=0, help="0 = the workload's size")
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

    # random-access rates of this GPU (the random-sector roofline's denominators)
    rates = binding.random_access_rates(gib=16, n_access=1 << 28)
    model = workload_model(args.workload)
    mode = binding.REACH_PERSISTENT if args.mode == "persistent" else binding.REACH_PER_LEVEL
    ctx = binding.ReachContext(LOG2_BUCKETS, model.state_words, max_levels=MAX_LEVELS,
                               line_buckets=args.line_buckets)
    ctx.load(model)
    stream = torch.cuda.current_stream()

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
            if mode == binding.REACH_PERSISTENT:
                pass
        e1.record(stream)
        torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / args.steps
    # the dominant kernel's device time, per launch (events recorded on the launch stream)
    kms = []
    for _ in range(3):
        ctx.run(mode)
        k, n = ctx.last_timing()
        kms.append(k)
        launches = n
    kernel_ms = sorted(kms)[1]
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

    peak, which = peaks()
    alg = algorithmic_bytes(got.states, got.transitions, model.state_words)
    achieved = alg / (kernel_ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "states/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": model.name, "states": got.states, "transitions": got.transitions,
                   "levels": len(got.level_sizes), "state_words": model.state_words,
                   "log2_buckets": LOG2_BUCKETS, "line_buckets": args.line_buckets,
                   "mode": args.mode, "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (4.3 GB table per step; bucket array 256 MiB)"},
        "find_or_put_ops_per_s": trans_all / (t_max / 1000.0),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_reach_persistent" if mode == 0 else "k_reach_level",
                     "kernel_ms": kernel_ms, "algorithmic_bytes": alg, "peak_source": which},
        "random_roofline": random_roofline(got.states, got.transitions, kernel_ms, rates, peak,
                                           model.state_words),
        "e2e": {"value": states_all / (e2e_ms / 1000.0), "unit": "states/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches * args.steps,
        "clocks": clocks.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(model)
        line["cpu_baseline"]["host_cores_available"] = os.cpu_count()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
