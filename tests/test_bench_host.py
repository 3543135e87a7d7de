"""Host-side logic of bench.py (no GPU): the multi-rank reduction over gloo,
the roofline arithmetic, the clock-sample parser and the reference arm."""
import json
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    step_ms = [12.5, 20.0][rank]          # rank 1 is the slow one
    states = [100.0, 300.0][rank]
    t = bench.max_over_ranks(step_ms, world)
    s = bench.sum_over_ranks(states, world)
    bench.barrier(world)
    q.put((rank, t, s))
    dist.destroy_process_group()


def test_two_rank_reduction_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, s in out:
        assert t == 20.0        # the job takes as long as the slowest rank
        assert s == 400.0       # value counts every rank's units


def test_algorithmic_bytes_per_unit():
    # 1 expanded state, 1 duplicate and 1 new successor at W = 16:
    # states*(64+4) + dup*(32+64) + new*(64+64+4)
    assert bench.algorithmic_bytes(states=2, transitions=2, state_words=16) == 2 * 68 + 1 * 96 + 1 * 132
    # rows are padded to 16 bytes
    assert bench.algorithmic_bytes(2, 2, 5) == bench.algorithmic_bytes(2, 2, 8)


def test_random_roofline_arithmetic():
    rates = {0: 1e9, 1: 5e8, 2: 1e9, 3: 1e9}
    r = bench.random_roofline(states=11, transitions=20, kernel_ms=1.0, rates=rates, hbm_gbs=1.0,
                              state_words=16)
    # 20 sector reads, 10 row reads, 3*10 writes at the probe rates, 2*11*64 B streamed at 1 GB/s
    want_s = 20 / 1e9 + 10 / 5e8 + 30 / 1e9 + 2 * 11 * 64 / 1e9
    assert abs(r["bound_ms"] - want_s * 1e3) < 1e-12
    assert abs(r["frac"] - want_s * 1e3) < 1e-12


def test_random_bound_scales_with_row_width():
    rates = {0: 1e9, 1: 5e8, 2: 1e9, 3: 1e9}
    # 32-byte rows (W <= 8): the compare is one 32 B read, a new state two sector writes
    got = bench.random_bound_s(states=11, transitions=20, rates=rates, hbm_gbs=1.0, state_words=8)
    assert abs(got - (20 / 1e9 + 10 / 1e9 + 2 * 10 / 1e9 + 2 * 11 * 32 / 1e9)) < 1e-15
    # 128-byte rows (W = 32): two 64 B reads per compare, five sector writes per new state
    got = bench.random_bound_s(states=11, transitions=20, rates=rates, hbm_gbs=1.0, state_words=32)
    assert abs(got - (20 / 1e9 + 10 * 2 / 5e8 + 5 * 10 / 1e9 + 2 * 11 * 128 / 1e9)) < 1e-15


def test_clock_summary_parses_nvidia_smi_lines():
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Active",
               "0, 1980, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s["sm_max_mhz"] == 2070.0 and s["samples"] == 2
    assert s["reasons"] == ["sw_power_cap"]
    # the wider query: memory clock, temperature and bus id as medians / last seen
    c.lines = ["0, 2070, 2070, 441.2, 0x0, Not Active, Not Active, Not Active, Not Active, 3996, 30, 0:07.0",
               "0, 2070, 2070, 460.0, 0x0, Not Active, Not Active, Not Active, Not Active, 3996, 31, 0:07.0",
               "0, 2070, 2070, 455.5, 0x0, Not Active, Not Active, Not Active, Not Active, [N/A], 32, 0:07.0"]
    s = c.summary()
    assert s["reasons"] == [] and s["samples"] == 3
    assert (s["power_w"], s["mem_mhz"], s["temp_c"], s["pci_bus_id"]) == (455.5, 3996.0, 31.0, "0:07.0")


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, BENCH_REF_SAMPLE="20000")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "states/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_recorded_traffic_only_for_the_same_kernel_sources(monkeypatch):
    sha = bench.kernel_sources_sha("k_reach_persistent")
    assert len(sha) == 16 and sha != bench.kernel_sources_sha("k_reach_batch")
    rec = {"unit": "transition", "bytes_per_unit": 100.0, "sources_sha": sha, "capture": "x"}
    monkeypatch.setattr(bench, "RECORDED_TRAFFIC", {"k_reach_persistent:w": rec})
    t, src = bench.recorded_traffic("k_reach_persistent:w", 10)
    assert t == 1000.0 and src["bytes_per_unit"] == 100.0
    # another workload of the same kernel: null, with the capture shown for reference
    t, src = bench.recorded_traffic("k_reach_persistent:other", 10)
    assert t is None and "k_reach_persistent:w" in src["smaller_workload_captures"]
    # sources changed since the capture: null
    monkeypatch.setattr(bench, "RECORDED_TRAFFIC",
                        {"k_reach_persistent:w": dict(rec, sources_sha="0" * 16)})
    t, src = bench.recorded_traffic("k_reach_persistent:w", 10)
    assert t is None and "changed" in src["note"]
