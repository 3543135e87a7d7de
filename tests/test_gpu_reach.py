"""Reachability on the GPU against the oracle (through the C ABI).

Bar: bit-exact states, transitions, deadlocks, per-level sizes and digest,
plus the table invariants after every run (done buckets = states, no bucket
left in the write state, table-scan digest = reported digest).
"""
import numpy as np
import pytest

import oracle
from conftest import hand_models, load_golden
from paper_1004_2772_gb300 import synth
from test_oracle_pins import TINY_BEEM

pytestmark = pytest.mark.gpu

MODES = [0, 1, 2]  # REACH_PERSISTENT, REACH_PER_LEVEL, REACH_GRAPH


def log2_for(states, lf=0.5):
    return max(6, int(np.ceil(np.log2(max(states, 1) / lf))))


def check(b, ctx, m, mode, ref=None):
    ref = ref or oracle.reach(m)
    got = ctx.reach(m, mode=mode)
    assert got.status == b.HT_OK
    assert got.states == ref.states
    assert got.transitions == ref.transitions
    assert got.deadlocks == ref.deadlocks
    assert got.level_sizes == ref.level_sizes
    assert got.digest == ref.digest
    done, writing, digest = ctx.scan()
    assert (done, writing, digest) == (ref.states, 0, ref.digest)
    return got


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L", [8, 16, 32])
def test_tiny_interleaving(cuda_lib, mode, L):
    m = synth.tiny_interleaving_model()
    ctx = cuda_lib.ReachContext(18, 5, max_levels=256, line_buckets=L)
    got = check(cuda_lib, ctx, m, mode)
    assert got.states == 100000 and got.transitions == 1000000


@pytest.mark.parametrize("mode", MODES)
def test_hand_models(cuda_lib, mode):
    ctx = cuda_lib.ReachContext(8, 8, max_levels=64)
    for m, d in hand_models():
        got = check(cuda_lib, ctx, m, mode)
        assert got.states == d["states"] and got.level_sizes == d["level_sizes"]


@pytest.mark.parametrize("kw", TINY_BEEM, ids=[f"seed{k['seed']}" for k in TINY_BEEM])
def test_tiny_guarded_models(cuda_lib, kw):
    m = synth.beem_shaped_model(**kw)
    ctx = cuda_lib.ReachContext(12, m.state_words, max_levels=1024)
    for mode in MODES:
        check(cuda_lib, ctx, m, mode)


@pytest.mark.parametrize("k", [3, 17, 42, 101, 200, 256])
def test_batched_family_models(cuda_lib, k):
    """Interleaving models with 8-32 words per state (every row shape)."""
    m = [x for x in synth.batched_models(count=1, first_seed=k, lo=1e3, hi=2e5)][0]
    ref = oracle.reach(m)
    ctx = cuda_lib.ReachContext(log2_for(ref.states), m.state_words, max_levels=4096)
    check(cuda_lib, ctx, m, 0, ref)


@pytest.mark.parametrize("W", [13, 16, 24, 32])
def test_guarded_model_row_shapes(cuda_lib, W):
    m = synth.beem_shaped_model(3, n_procs=8, n_shared=3, state_words=W, n_lo=3, n_hi=5,
                                update_pct=40)
    ref = oracle.reach(m, max_states=3_000_000)
    assert not ref.truncated
    ctx = cuda_lib.ReachContext(log2_for(ref.states), W, max_levels=4096)
    for mode in MODES:
        check(cuda_lib, ctx, m, mode, ref)


@pytest.mark.parametrize("W", [13, 16, 20, 24, 28, 32])
def test_guarded_model_every_row_width(cuda_lib, W):
    """A guarded model of 60,837 states and 35 levels with rows of 4 to 8
    16-byte chunks (every compiled row width from 13 words up), in all three
    drivers: many warp rounds per level and a table of 2^17 buckets (two
    blocks per SM)."""
    m = synth.beem_shaped_model(13, n_procs=10, n_shared=3, state_words=W, n_lo=3, n_hi=6,
                                update_pct=40)
    ref = oracle.reach(m)
    assert ref.states == 60837
    ctx = cuda_lib.ReachContext(log2_for(ref.states), W, max_levels=4096)
    for mode in MODES:
        check(cuda_lib, ctx, m, mode, ref)


@pytest.mark.parametrize("P,W", [(16, 16), (24, 24), (31, 32)])
def test_rounds_with_more_successors_than_descriptors(cuda_lib, P, W):
    """Every state has 2P successors (32, 48 or 62); a round holds
    min(32, 1920 / (2P)) states (the per-lane descriptor slices of the
    worst-case fan-out in the warp's 1920 descriptors): 32, 32 and 30.
    All three drivers, and tracing."""
    m = synth.interleaving_model(11, [2] * P, W) if P <= 16 else \
        synth.interleaving_model(11, [2] * 12 + [1] * (P - 12), W)
    ref = oracle.reach(m)
    ctx = cuda_lib.ReachContext(log2_for(ref.states), W, max_levels=4096)
    for mode in MODES + [cuda_lib.REACH_PERSISTENT | cuda_lib.REACH_TRACE]:
        check(cuda_lib, ctx, m, mode, ref)


def _fan_model(k):
    """Six 4-state interleaving processes (4096 states, 12 successors each)
    and a seventh process with one local state and k parallel self-loops:
    every state has 12 + k successors, k of them itself."""
    base = synth.interleaving_model(5, [4] * 6, 8)
    edges = []
    for p in range(6):
        b0 = int(base.edge_begin[4 * p])
        ep = []
        for s in range(4):
            lo, hi = int(base.edge_begin[4 * p + s]), int(base.edge_begin[4 * p + s + 1])
            ep.append([(int(base.edge_dst[e]), -1, 0, -1, 0) for e in range(lo, hi)])
        assert b0 == 8 * p
        edges.append(ep)
    edges.append([[(0, -1, 0, -1, 0)] * k])
    return synth.build_model(f"fan-{12 + k}", [4] * 6 + [1], edges, 8)


@pytest.mark.parametrize("k", [100, 1000, 1908])
def test_rounds_of_few_states(cuda_lib, k):
    """Fan-outs of 112, 1012 and 1920 successors per state: a warp round
    holds 17, 1 and 1 states, and the last fills all 1920 descriptors."""
    m = _fan_model(k)
    ref = oracle.reach(m)
    assert (ref.states, ref.transitions) == (4096, 4096 * (12 + k))
    ctx = cuda_lib.ReachContext(14, 8, max_levels=4096)
    for mode in MODES:
        check(cuda_lib, ctx, m, mode, ref)


def test_fan_out_beyond_the_descriptor_area_is_refused(cuda_lib):
    """1921 successors per state do not fit one warp round: the model is
    refused before any launch."""
    ctx = cuda_lib.ReachContext(14, 8, max_levels=4096)
    with pytest.raises(cuda_lib.HtError) as e:
        ctx.load(_fan_model(1909))
    assert e.value.status == cuda_lib.HT_ERR_INVALID
    # the context still runs a model that fits
    m = _fan_model(100)
    check(cuda_lib, ctx, m, 0, oracle.reach(m))


def test_repeated_runs_and_reload(cuda_lib):
    ctx = cuda_lib.ReachContext(18, 16, max_levels=4096)
    a = synth.tiny_interleaving_model()
    b = synth.beem_shaped_model(4, n_procs=6, n_shared=2, state_words=10, update_pct=50)
    ra, rb = oracle.reach(a), oracle.reach(b)
    for _ in range(2):
        check(cuda_lib, ctx, a, 0, ra)
        check(cuda_lib, ctx, b, 0, rb)
        check(cuda_lib, ctx, a, 1, ra)


def test_table_too_small_reports_full(cuda_lib):
    m = synth.tiny_interleaving_model()
    ctx = cuda_lib.ReachContext(16, 5, max_levels=256)   # 65536 buckets < 10^5 states
    for mode in MODES:
        got = ctx.reach(m, mode=mode, raise_on_error=False)
        assert got.status == cuda_lib.HT_ERR_FULL
        done, writing, _ = ctx.scan()
        assert writing == 0 and done <= 65536


def test_level_capacity_reports_levels(cuda_lib):
    m = synth.tiny_interleaving_model()
    ctx = cuda_lib.ReachContext(18, 5, max_levels=5)
    for mode in MODES:
        got = ctx.reach(m, mode=mode, raise_on_error=False)
        assert got.status == cuda_lib.HT_ERR_LEVELS


def test_invalid_models_rejected(cuda_lib):
    m = synth.tiny_interleaving_model()
    ctx = cuda_lib.ReachContext(10, 8, max_levels=64)
    bad = synth.tiny_interleaving_model()
    bad.init = bad.init.copy()
    bad.init[0] = 10                      # local state out of range
    with pytest.raises(cuda_lib.HtError):
        ctx.load(bad)
    wide = synth.interleaving_model(1, [2] * 9, 9)   # 9 words > context maximum of 8
    with pytest.raises(cuda_lib.HtError):
        ctx.load(wide)
    bad2 = synth.tiny_interleaving_model()
    bad2.edge_dst = bad2.edge_dst.copy()
    bad2.edge_dst[3] = 99                 # edge target out of range
    with pytest.raises(cuda_lib.HtError):
        ctx.load(bad2)
    ctx.load(m)                           # a valid model still loads afterwards


def test_beem_shaped_medium(cuda_lib):
    """A guarded 12-process model of about a million states, both drivers."""
    g = load_golden("beem_medium.json")
    m = synth.beem_shaped_model(**g["model"])
    ctx = cuda_lib.ReachContext(g["log2_buckets"], 16, max_levels=4096)
    for mode in MODES:
        got = ctx.reach(m, mode=mode)
        assert (got.states, got.transitions, got.deadlocks, got.digest) == (
            g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
        assert got.level_sizes == g["level_sizes"]


def test_beem_shaped_workload_full_size(cuda_lib):
    """The benchmarked BEEM-shaped workload (32M states, 2^26 buckets), in the
    launch configuration bench.py times, against the oracle's stored result."""
    g = load_golden("beem_c2.json")
    m = synth.beem_shaped_model(**g["model"])
    ctx = cuda_lib.ReachContext(g["log2_buckets"], 16, max_levels=1 << 14)
    got = ctx.reach(m, mode=0)
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
    assert got.level_sizes == g["level_sizes"]
    done, writing, digest = ctx.scan()
    assert (done, writing, digest) == (g["states"], 0, int(g["digest"], 16))


def _min_deadlock_level(m, ref):
    """Lowest BFS level holding a state without successors (oracle states in
    discovery order, which is level order)."""
    r = oracle.reach(m, keep_states=True, keep_cap=1 << 21)
    start = 0
    for lvl, size in enumerate(ref.level_sizes):
        if start + size > r.state_list.shape[0]:
            return None
        for s in r.state_list[start:start + size]:
            if oracle.successors(m, s).shape[0] == 0:
                return lvl
        start += size
    return None


def _check_trace(m, level, path, ref):
    assert level == _min_deadlock_level(m, ref)
    assert path.shape[0] == level + 1
    assert np.array_equal(path[0], m.init)
    for a, b in zip(path[:-1], path[1:]):
        succ = oracle.successors(m, a)
        assert any(np.array_equal(b, x) for x in succ), "consecutive trace states are not a transition"
    assert oracle.successors(m, path[-1]).shape[0] == 0


@pytest.mark.parametrize("which", ["deadlock-chain", "tiny0", "tiny1", "tiny2", "medium"])
def test_deadlock_trace(cuda_lib, which):
    if which == "deadlock-chain":
        m = [m for m, d in hand_models() if d["name"] == which][0]
        lg = 8
    elif which == "medium":
        g = load_golden("beem_medium.json")
        m = synth.beem_shaped_model(**g["model"])
        lg = g["log2_buckets"]
    else:
        kws = [kw for kw in TINY_BEEM if oracle.reach(synth.beem_shaped_model(**kw)).deadlocks > 0]
        m = synth.beem_shaped_model(**kws[int(which[-1])])
        lg = 12
    ref = oracle.reach(m)
    assert ref.deadlocks > 0
    ctx = cuda_lib.ReachContext(lg, m.state_words, max_levels=4096)
    got = ctx.reach(m, mode=cuda_lib.REACH_PERSISTENT | cuda_lib.REACH_TRACE)
    assert (got.states, got.transitions, got.deadlocks, got.digest, got.level_sizes) == (
        ref.states, ref.transitions, ref.deadlocks, ref.digest, ref.level_sizes)
    level, path = ctx.deadlock_trace()
    _check_trace(m, level, path, ref)


@pytest.mark.parametrize("which", ["tiny0", "medium"])
def test_deadlock_trace_16_bit_buckets(cuda_lib, which):
    """Tracing with 16-bit buckets (its default 16-bucket line): the same
    shortest-path trace properties, and the run itself bit-exact."""
    if which == "medium":
        g = load_golden("beem_medium.json")
        m = synth.beem_shaped_model(**g["model"])
        lg = g["log2_buckets"]
    else:
        kws = [kw for kw in TINY_BEEM if oracle.reach(synth.beem_shaped_model(**kw)).deadlocks > 0]
        m = synth.beem_shaped_model(**kws[0])
        lg = 12
    ref = oracle.reach(m)
    assert ref.deadlocks > 0
    ctx = cuda_lib.ReachContext(lg, m.state_words, max_levels=4096, bucket_bits=16)
    got = ctx.reach(m, mode=cuda_lib.REACH_PERSISTENT | cuda_lib.REACH_TRACE)
    assert (got.states, got.transitions, got.deadlocks, got.digest, got.level_sizes) == (
        ref.states, ref.transitions, ref.deadlocks, ref.digest, ref.level_sizes)
    level, path = ctx.deadlock_trace()
    _check_trace(m, level, path, ref)


@pytest.mark.parametrize("which", ["tiny1", "medium"])
def test_deadlock_trace_prime_line_table(cuda_lib, which):
    """Tracing in a table of a prime number of 32-bucket lines (division by
    the line count instead of a mask): 131 lines for a tiny guarded model,
    2^19 - 1 lines (load 0.33) for the medium model."""
    if which == "medium":
        m = synth.beem_shaped_model(**load_golden("beem_medium.json")["model"])
        lines = (1 << 19) - 1
    else:
        kws = [kw for kw in TINY_BEEM if oracle.reach(synth.beem_shaped_model(**kw)).deadlocks > 0]
        m = synth.beem_shaped_model(**kws[1])
        lines = 131
    ref = oracle.reach(m)
    ctx = cuda_lib.ReachContext(None, m.state_words, n_buckets=32 * lines, max_levels=4096)
    got = ctx.reach(m, mode=cuda_lib.REACH_PERSISTENT | cuda_lib.REACH_TRACE)
    assert (got.states, got.transitions, got.deadlocks, got.digest, got.level_sizes) == (
        ref.states, ref.transitions, ref.deadlocks, ref.digest, ref.level_sizes)
    level, path = ctx.deadlock_trace()
    _check_trace(m, level, path, ref)


def test_no_deadlock_no_trace(cuda_lib):
    m = synth.tiny_interleaving_model()
    ctx = cuda_lib.ReachContext(18, 5, max_levels=256)
    ctx.reach(m, mode=cuda_lib.REACH_PERSISTENT | cuda_lib.REACH_TRACE)
    level, path = ctx.deadlock_trace()
    assert level is None and path.shape[0] == 0


def test_run_times_ring(cuda_lib):
    """Every launch of a loop keeps its own kernel time (no sync inside the loop)."""
    m = synth.tiny_interleaving_model()
    ctx = cuda_lib.ReachContext(18, 5, max_levels=256)
    ctx.load(m)
    for _ in range(70):                   # more runs than the ring keeps
        ctx.run(cuda_lib.REACH_PERSISTENT)
    t = ctx.run_times(100)
    assert t.shape[0] == 64 and (t > 0).all()
    assert abs(float(t[-1]) - ctx.last_timing()[0]) < 1e-6
    assert ctx.result().states == 100000


def _stored_rows(b, ctx, W):
    """The state vectors held by the done buckets of a context's table."""
    import torch
    bk, d, rw = b.ht_arrays(ctx.table_handle())
    base = ctx.mem.data_ptr()
    nb = ctx.n_buckets
    torch.cuda.synchronize()
    words = ctx.mem[bk - base:bk - base + 4 * nb].view(torch.int32).cpu().numpy()
    rows = ctx.mem[d - base:d - base + 4 * nb * rw].view(torch.int32).view(nb, rw).cpu().numpy()
    done = (words.view(np.uint32) >> 31) == 1
    return rows[done][:, :W]


def _sorted_rows(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a[np.lexsort(a.T[::-1])]


@pytest.mark.parametrize("which", ["tiny", "guarded", "batched", "medium"])
def test_stored_set_is_exactly_the_reachable_set(cuda_lib, which):
    """The invariants beyond the counts: the done buckets hold pairwise
    distinct vectors, and these are exactly the states the oracle's BFS
    enumerates (nothing unreachable stored, nothing reachable missing)."""
    if which == "tiny":
        m = synth.tiny_interleaving_model()
    elif which == "guarded":
        m = synth.beem_shaped_model(3, n_procs=9, update_pct=40)        # 3,011 states, 80 deadlocks
    elif which == "batched":
        m = synth.batched_models(count=1, first_seed=17, lo=1e3, hi=2e5)[0]
    else:
        m = synth.beem_shaped_model(**load_golden("beem_medium.json")["model"])  # 5.5M states
    ref = oracle.reach(m, keep_states=True, keep_cap=1 << 23)
    assert not ref.truncated and ref.state_list.shape[0] == ref.states
    ctx = cuda_lib.ReachContext(log2_for(ref.states), m.state_words, max_levels=4096)
    for mode in MODES:
        check(cuda_lib, ctx, m, mode, ref)
        got = _sorted_rows(_stored_rows(cuda_lib, ctx, m.state_words))
        assert got.shape == (ref.states, m.state_words)
        assert not (got[1:] == got[:-1]).all(axis=1).any()          # no vector stored twice
        assert np.array_equal(got, _sorted_rows(ref.state_list))   # the reachable set itself


@pytest.mark.parametrize("seed", [1, 0x9E3779B97F4A7C15, (1 << 64) - 1])
def test_results_do_not_depend_on_the_hash_seed(cuda_lib, seed):
    """The hash seed moves every state to other buckets (other lines, other
    walks, other claim races); the visited set, the counts, the level sizes
    and the digest must not move with it.  A guarded model in all three
    drivers, and the table's contents must be the same set."""
    m = synth.beem_shaped_model(13, n_procs=10, n_shared=3, state_words=16, n_lo=3, n_hi=6,
                                update_pct=40)
    ref = oracle.reach(m)
    ctx = cuda_lib.ReachContext(17, 16, max_levels=4096, hash_seed=seed)
    for mode in MODES:
        check(cuda_lib, ctx, m, mode, ref)
