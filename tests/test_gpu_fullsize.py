"""The batched and served configurations at their full sizes against stored
expected values (tests/golden/batched_256.json, served_seed5.json).

Those values come from the closed forms of the interleaving family and the CPU
oracle (tests/golden/make_golden.py); nothing in them comes from the GPU.
Every model's states, transitions, deadlocks, level sizes and set digest must
match bit-exactly (Alg. "Reachability analysis": the set of reachable states
and its BFS levels do not depend on how the work is scheduled).

* batched: the 256 models of uneven size (3-12 processes, 8-32 words,
  10^3-10^6 states each) in one persistent launch under a CUDA graph, with the
  default size estimates and table growth -- the launch bench.py times --
  captured once and replayed;
* served: the Poisson stream of 180 jobs of 10^4 to 2*10^8 states (64-byte
  states) through a 64-slot server with the HBM budget bench.py uses, once
  with every job queued at once (the many-job continuous-batching kernel) and
  once in real-time arrival order (jobs that find the GPU idle run on the
  single-model kernel).
"""
import time

import pytest

from conftest import load_golden
from paper_1004_2772_gb300 import synth

pytestmark = pytest.mark.gpu


def _same(got, e, what):
    assert got.status == 0, (what, got.status)
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        e["states"], e["transitions"], e["deadlocks"], int(e["digest"], 16)), what
    assert got.level_sizes == e["level_sizes"], what


def test_batched_256_models_full_size(cuda_lib):
    g = load_golden("batched_256.json")
    models = synth.batched_models(count=256, first_seed=1)
    assert [m.name for m in models] == [e["name"] for e in g["models"]]
    b = cuda_lib.ReachBatch(models, max_levels=4096)
    for rep in range(2):  # capture, then replay of the same graph
        b.run(use_graph=True)
        res, grows, st = b.results()
        assert st == 0
        for m, got, e in zip(models, res, g["models"]):
            _same(got, e, (rep, m.name))
    assert sum(grows) > 0  # the default estimates make tables grow
    b.close()


def _drain(srv, n, timeout_s):
    got = {}
    t0 = time.time()
    while len(got) < n:
        for j in srv.poll():
            got[j.job_id] = j
        assert time.time() - t0 < timeout_s, f"only {len(got)} of {n} jobs finished"
        time.sleep(0.001)
    return got


@pytest.fixture(scope="module")
def served():
    g = load_golden("served_seed5.json")
    jobs = synth.served_jobs(seed=5, rate=20.0, duration_s=10.0)
    assert [m.name for _, m in jobs] == [e["name"] for e in g["jobs"]]
    return jobs, g["jobs"]


def _server(cuda_lib):
    import gc

    import torch
    # the previous server's arena goes back to the driver first: the budget is
    # a share of what the device has free
    gc.collect()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    return cuda_lib.Server(budget_bytes=int(free * 0.85), n_slots=64, max_levels=4096)


def test_served_stream_full_size_all_queued(cuda_lib, served):
    jobs, want = served
    srv = _server(cuda_lib)
    ids = [srv.submit(m) for _, m in jobs]
    st = srv.status()
    assert st["queued"] + st["running"] >= 8  # a real queue: the many-job kernel serves it
    got = _drain(srv, len(ids), timeout_s=900)
    for jid, (_, m), e in zip(ids, jobs, want):
        _same(got[jid].result, e, m.name)
    srv.close()
    del srv


def test_served_stream_full_size_real_time(cuda_lib, served):
    jobs, want = served
    srv = _server(cuda_lib)
    ids, got, k, t0 = [], {}, 0, time.time()
    while len(got) < len(jobs):
        now = time.time() - t0
        while k < len(jobs) and jobs[k][0] <= now:
            ids.append(srv.submit(jobs[k][1]))
            k += 1
        for j in srv.poll():
            got[j.job_id] = j
        assert now < 900, f"only {len(got)} of {len(jobs)} jobs finished"
        time.sleep(0.0005)
    for jid, (_, m), e in zip(ids, jobs, want):
        _same(got[jid].result, e, m.name)
    assert srv.status()["kernel_launches"] >= 1
    srv.close()
    del srv
