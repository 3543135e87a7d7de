"""Batched reachability (one persistent launch, many models) against the oracle.

Every model's result in the batch must be bit-identical to the oracle's for
that model alone: states, transitions, deadlocks, level sizes and digest --
whatever the interleaving with the other models, whether tables had to grow,
and whether the batch ran as a plain launch or as a replayed CUDA graph.
"""
import numpy as np
import pytest

import oracle
from conftest import load_golden
from paper_1004_2772_gb300 import synth
from test_oracle_pins import TINY_BEEM

pytestmark = pytest.mark.gpu


def _same(got, ref, what=""):
    assert got.status == 0, what
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        ref.states, ref.transitions, ref.deadlocks, ref.digest), what
    assert got.level_sizes == ref.level_sizes, what


@pytest.fixture(scope="module")
def family():
    models = synth.batched_models(count=24, first_seed=1, lo=1e3, hi=4e4)
    refs = [oracle.reach(m) for m in models]
    return models, refs


# The growth rule of the batch kernel, restated on the host: before a level,
# a table grows if the states stored so far plus the coming level's states
# times the model's fan-out bound (capped by the model's state bound, when it
# has one) exceed GROW_AT of its buckets.  The new size holds that estimate at
# load GROW_TO -- or the state bound itself, when there is one and its table
# still fits the pool.  Growth changes no result, only the table sizes; the
# tests use this to predict how often each model grows.
GROW_AT = float(np.float32(0.9))
GROW_TO = 0.5


def _maxfan(m):
    eb, tot, base = m.edge_begin, 0, 0
    for p in range(m.n_procs):
        n = int(m.n_local[p])
        tot += max(int(eb[base + s + 1] - eb[base + s]) for s in range(n))
        base += n
    return tot


def _growth_path(cuda_lib, level_sizes, maxfan, bound, lg0, state_words, pool_free):
    """Table sizes (log2) a model grows through, and "ok" or "oom"."""
    lg, used, path, stored = lg0, 0, [], 1
    for k in range(len(level_sizes) - 1):
        n_next = level_sizes[k + 1]
        stored += n_next
        need = float(stored) + float(n_next) * maxfan
        if bound:
            need = min(need, float(bound))
        if need <= GROW_AT * (1 << lg):
            continue

        def size_for(x):
            s = lg + 1
            while s < 31 and (1 << s) * GROW_TO < x:
                s += 1
            return s

        nl = size_for(need)
        if bound:
            nlb = size_for(float(bound))
            if nlb > nl and used + cuda_lib.generation_bytes(nlb, state_words) <= pool_free:
                nl = nlb
        b = cuda_lib.generation_bytes(nl, state_words)
        if used + b > pool_free:
            return path, "oom"
        used += b
        lg = nl
        path.append(nl)
    return path, "ok"


def test_batch_matches_oracle_with_growth(cuda_lib, family):
    models, refs = family
    # start every table at 2^10 buckets so that most of them must grow; with
    # room in the pool, a model with a state bound grows once, to the bound
    b = cuda_lib.ReachBatch(models, log2_initial=[10] * len(models), max_levels=1024)
    b.run(use_graph=False)
    res, grows, st = b.results()
    assert st == 0
    for m, got, ref, gr in zip(models, res, refs, grows):
        _same(got, ref, m.name)
        path, _ = _growth_path(cuda_lib, ref.level_sizes, _maxfan(m), int(np.prod(m.n_local)), 10,
                               m.state_words, 1 << 60)
        assert gr == len(path) <= 1, m.name
    assert sum(grows) > 0


@pytest.mark.parametrize("seed", [50, 51, 58])
def test_batch_growth_without_room_for_the_bound(cuda_lib, seed):
    """A pool too small for the bound's table: the model grows step by step
    from its level estimates (or runs out of pool, reported as HT_ERR_OOM),
    exactly as the host restatement of the rule predicts."""
    m = synth.batched_models(count=1, first_seed=seed, lo=2e4, hi=2e5)[0]
    ref = oracle.reach(m)
    bound = int(np.prod(m.n_local))
    final = 10
    while (1 << final) * GROW_TO < bound:
        final += 1
    free = cuda_lib.generation_bytes(final, m.state_words) - 256
    path, outcome = _growth_path(cuda_lib, ref.level_sizes, _maxfan(m), bound, 10, m.state_words, free)
    b = cuda_lib.ReachBatch([m], log2_initial=[10], max_levels=1024,
                            pool_bytes=cuda_lib.generation_bytes(10, m.state_words) + free)
    b.run(use_graph=False)
    res, grows, st = b.results()
    assert int(grows[0]) == len(path)
    if outcome == "ok":
        assert st == 0 and len(path) >= 2
        _same(res[0], ref, m.name)
    else:
        assert st == cuda_lib.HT_ERR_OOM and res[0].status == cuda_lib.HT_ERR_OOM


def test_batch_unbounded_model_grows_step_by_step(cuda_lib):
    """A guarded model with shared variables has no state bound: its table
    grows through the sizes the level estimates give, and the result is the
    oracle's."""
    g = load_golden("beem_medium.json")
    m = synth.beem_shaped_model(**g["model"])
    path, outcome = _growth_path(cuda_lib, g["level_sizes"], _maxfan(m), 0, 10, m.state_words, 1 << 60)
    assert outcome == "ok" and len(path) >= 3
    pool = sum(cuda_lib.generation_bytes(lg, m.state_words) for lg in [10] + path) + 4096
    b = cuda_lib.ReachBatch([m], log2_initial=[10], max_levels=4096, pool_bytes=pool)
    b.run(use_graph=False)
    res, grows, st = b.results()
    assert st == 0 and int(grows[0]) == len(path)
    got = res[0]
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
    assert got.level_sizes == g["level_sizes"]


def test_batch_graph_replay_is_identical(cuda_lib, family):
    models, refs = family
    b = cuda_lib.ReachBatch(models, max_levels=1024)   # default estimates
    for _ in range(3):
        b.run(use_graph=True)
        res, grows, st = b.results()
        assert st == 0
        for m, got, ref in zip(models, res, refs):
            _same(got, ref, m.name)


def test_batch_mixed_shapes_and_guards(cuda_lib):
    """Guarded models with shared variables (no state bound: growth is sized
    from the fan-out bound) mixed with interleaving models of 8..32 words."""
    models = [synth.beem_shaped_model(**kw) for kw in TINY_BEEM[:6]]
    models += synth.batched_models(count=6, first_seed=200, lo=5e2, hi=2e4)
    models.append(synth.tiny_interleaving_model())
    refs = [oracle.reach(m) for m in models]
    b = cuda_lib.ReachBatch(models, log2_initial=[10] * len(models), max_levels=1024)
    b.run(use_graph=True)
    res, grows, st = b.results()
    for m, got, ref in zip(models, res, refs):
        _same(got, ref, m.name)


def test_batch_equals_single_model_runs(cuda_lib, family):
    models, refs = family
    one = []
    for m in models[:6]:
        ctx = cuda_lib.ReachContext(18, m.state_words, max_levels=1024)
        one.append(ctx.reach(m))
        ctx.close()
    b = cuda_lib.ReachBatch(models[:6], max_levels=1024)
    b.run()
    res, _, st = b.results()
    assert st == 0
    for a, c in zip(res, one):
        assert (a.states, a.transitions, a.digest, a.level_sizes) == (
            c.states, c.transitions, c.digest, c.level_sizes)


def test_batch_pool_exhaustion_is_reported(cuda_lib):
    models = synth.batched_models(count=4, first_seed=50, lo=2e4, hi=4e4)
    refs = [oracle.reach(m) for m in models]
    init = sum(cuda_lib.generation_bytes(10, m.state_words) for m in models)
    b = cuda_lib.ReachBatch(models, log2_initial=[10] * 4, max_levels=1024, pool_bytes=init + 4096)
    b.run(use_graph=False)
    res, grows, st = b.results()
    assert st == cuda_lib.HT_ERR_OOM
    assert all(r.status in (0, cuda_lib.HT_ERR_OOM) for r in res)
    for got, ref in zip(res, refs):
        if got.status == 0:
            assert got.states == ref.states
