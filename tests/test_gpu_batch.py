"""Batched reachability (one persistent launch, many models) against the oracle.

Every model's result in the batch must be bit-identical to the oracle's for
that model alone: states, transitions, deadlocks, level sizes and digest --
whatever the interleaving with the other models, whether tables had to grow,
and whether the batch ran as a plain launch or as a replayed CUDA graph.
"""
import pytest

import oracle
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


def test_batch_matches_oracle_with_growth(cuda_lib, family):
    models, refs = family
    # start every table at 2^10 buckets so that most of them must grow
    b = cuda_lib.ReachBatch(models, log2_initial=[10] * len(models), max_levels=1024)
    b.run(use_graph=False)
    res, grows, st = b.results()
    assert st == 0
    for m, got, ref in zip(models, res, refs):
        _same(got, ref, m.name)
    assert sum(grows) > 0 and max(grows) >= 2


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
