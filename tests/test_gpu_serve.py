"""Served reachability (continuous batching) against the oracle and against
each job run alone.

Jobs are admitted into slots of one running kernel as slots and memory free
up; their levels overlap on the device.  Every job's result must be the same
as the oracle's and as reach() on that job alone (tolerance 0: the results are
integers and a digest).
"""
import time

import pytest

import oracle
from paper_1004_2772_gb300 import synth

pytestmark = pytest.mark.gpu


def _drain(srv, n, timeout_s=60.0):
    got = {}
    t0 = time.time()
    while len(got) < n:
        for j in srv.poll():
            got[j.job_id] = j
        assert time.time() - t0 < timeout_s, f"only {len(got)} of {n} jobs finished"
        time.sleep(0.001)
    return got


def _same(r, ref):
    assert r.status == 0
    assert (r.states, r.transitions, r.deadlocks, r.digest) == (
        ref.states, ref.transitions, ref.deadlocks, ref.digest)
    assert r.level_sizes == ref.level_sizes


@pytest.fixture(scope="module")
def jobs():
    js = synth.served_jobs(seed=3, rate=1000.0, duration_s=1.0, lo=1e3, hi=5e4, max_jobs=14)
    models = [m for _, m in js]
    return models, [oracle.reach(m) for m in models]


def test_served_jobs_equal_oracle_and_alone(cuda_lib, jobs):
    models, refs = jobs
    alone = []
    for m in models:
        ctx = cuda_lib.ReachContext(18, m.state_words, max_levels=2048)
        alone.append(ctx.reach(m))
        ctx.close()
    srv = cuda_lib.Server(budget_bytes=2 << 30, n_slots=4, max_levels=2048)
    ids = [srv.submit(m) for m in models]          # more jobs than slots: some wait
    got = _drain(srv, len(ids))
    for jid, ref, a in zip(ids, refs, alone):
        r = got[jid].result
        _same(r, ref)
        assert (r.states, r.transitions, r.digest, r.level_sizes) == (
            a.states, a.transitions, a.digest, a.level_sizes)
    srv.close()


def test_admission_waits_for_memory(cuda_lib, jobs):
    models, refs = jobs
    # room for about two of these jobs at a time
    per_job = max(cuda_lib.generation_bytes(17, m.state_words) for m in models[:6])
    srv = cuda_lib.Server(budget_bytes=int(2.5 * per_job), n_slots=8, max_levels=2048)
    ids = [srv.submit(m, log2_buckets=17) for m in models[:6]]
    st = srv.status()
    assert st["queued"] >= 3 and st["running"] <= 2
    got = _drain(srv, len(ids))
    for jid, ref in zip(ids, refs[:6]):
        _same(got[jid].result, ref)
    # a job that can never fit is refused, the server keeps working
    big = synth.sized_interleaving_model(1, 6, 16, 10**7)
    bad = srv.submit(big)
    ok = srv.submit(models[0])
    got = _drain(srv, 2)
    assert got[bad].result.status == cuda_lib.HT_ERR_OOM
    _same(got[ok].result, refs[0])
    srv.close()


def test_staggered_arrivals_and_kernel_restart(cuda_lib, jobs):
    models, refs = jobs
    srv = cuda_lib.Server(budget_bytes=2 << 30, n_slots=3, max_levels=2048)
    ids = []
    for m in models[:8]:
        ids.append(srv.submit(m))
        time.sleep(0.002)                          # arrivals while others run
        srv.poll(max_done=0)
    got = _drain(srv, len(ids))
    time.sleep(0.5)                                # idle: the kernel leaves on its own
    late = srv.submit(models[8])
    got.update(_drain(srv, 1))
    for jid, ref in zip(ids + [late], refs[:8] + [refs[8]]):
        _same(got[jid].result, ref)
    assert srv.status()["kernel_launches"] >= 2
    srv.close()


def test_lone_jobs_on_idle_server_guarded_and_full(cuda_lib):
    """Jobs that find the GPU idle run on the single-model kernel: a guarded
    model (shared variables, table size given), a table too small for its job
    (HT_ERR_FULL, the server keeps serving), then a burst that goes to the
    many-job kernel."""
    from test_oracle_pins import TINY_BEEM
    srv = cuda_lib.Server(budget_bytes=1 << 30, n_slots=4, max_levels=2048)
    guarded = synth.beem_shaped_model(**TINY_BEEM[0])
    ref = oracle.reach(guarded)
    jid = srv.submit(guarded, log2_buckets=14)
    got = _drain(srv, 1)
    _same(got[jid].result, ref)
    small = synth.sized_interleaving_model(7, 4, 16, 20000)        # 20k states into 2^10 buckets
    jid = srv.submit(small, log2_buckets=10)
    got = _drain(srv, 1)
    assert got[jid].result.status == cuda_lib.HT_ERR_FULL
    burst = [synth.sized_interleaving_model(100 + k, 3 + k % 4, 16, 3000 + 700 * k) for k in range(6)]
    refs = [oracle.reach(m) for m in burst]
    ids = [srv.submit(m) for m in burst]
    got = _drain(srv, len(ids))
    for i, r in zip(ids, refs):
        _same(got[i].result, r)
    assert srv.status()["kernel_launches"] >= 3
    srv.close()
