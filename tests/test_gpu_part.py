"""Owner-partitioned reachability (part_reach_*: K owner partitions on one GPU,
successors exchanged between them every level) against the oracle.

States, transitions, deadlocks, level sizes and the set digest must be
bit-exact whatever the number of owners and the chunk size of the exchange;
the owners' state counts add up to the states; the exchanged count is the
successors whose owner is not their source; the device's exchange plan is
the layout paper_1004_2772_gb300.exchange.plan gives for the same counts (the
layout the cross-process exchange delivers).
"""
import numpy as np
import pytest

import oracle
from conftest import load_golden
from paper_1004_2772_gb300 import exchange, synth
from test_oracle_pins import TINY_BEEM

pytestmark = pytest.mark.gpu


def _same(got, ref, what=""):
    assert got.status == 0, what
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        ref.states, ref.transitions, ref.deadlocks, ref.digest), what
    assert got.level_sizes == ref.level_sizes, what


@pytest.mark.parametrize("K", [2, 4])
def test_beem_shaped_full_size(cuda_lib, K):
    g = load_golden("beem_c2.json")
    m = synth.beem_shaped_model(**g["model"])
    lg = 26 - K.bit_length() + 1
    pr = cuda_lib.PartReach(K, lg, m.state_words)
    got, parts, ex = pr.run(m)
    assert got.status == 0
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
    assert got.level_sizes == g["level_sizes"]
    assert sum(parts) == got.states and min(parts) > 0.9 * got.states / K
    # owners are hash bits: a successor other than its parent changes
    # partition with probability (K - 1) / K; one equal to its parent (a
    # self-loop, or an update writing the value already there) never does
    frac = ex / got.transitions
    assert 0.85 * (K - 1) / K < frac <= (K - 1) / K + 0.01
    pr.close()


@pytest.mark.parametrize("K", [1, 2, 4, 8, 16])
def test_tiny_any_owner_count(cuda_lib, K):
    m = synth.tiny_interleaving_model()
    ref = oracle.reach(m)
    pr = cuda_lib.PartReach(K, max(10, 18 - K.bit_length() + 1), m.state_words)
    got, parts, ex = pr.run(m)
    _same(got, ref, K)
    assert sum(parts) == ref.states
    assert (ex == 0) == (K == 1)
    pr.close()


def test_guarded_models(cuda_lib):
    """Guarded models (shared variables, updates, mutex), brute-force pinned."""
    for kw in TINY_BEEM:
        m = synth.beem_shaped_model(**kw)
        ref = oracle.reach(m)
        for K in (2, 4):
            pr = cuda_lib.PartReach(K, 10, m.state_words)
            got, parts, _ = pr.run(m)
            _same(got, ref, (m.name, K))
            assert sum(parts) == ref.states
            pr.close()


def test_small_exchange_chunks(cuda_lib):
    """The smallest exchange chunk (960 rows: one warp round of successors per
    chunk) splits every level of a guarded model into many chunks."""
    m = synth.beem_shaped_model(13, n_procs=10, n_shared=3, state_words=16, n_lo=3, n_hi=6, update_pct=40)
    ref = oracle.reach(m)
    assert ref.states > 50_000
    for K in (1, 4):
        pr = cuda_lib.PartReach(K, 17 - K.bit_length() + 1, m.state_words, exchange_rows=960)
        got, _, _ = pr.run(m)
        _same(got, ref, K)
        pr.close()


def test_wide_rows(cuda_lib):
    """Rows of 8..32 words (the compiled row widths 2, 4 and 8 chunks)."""
    for m in synth.batched_models(count=6, first_seed=300, lo=2e3, hi=3e4):
        ref = oracle.reach(m)
        pr = cuda_lib.PartReach(4, 14, m.state_words)
        got, parts, _ = pr.run(m)
        _same(got, ref, m.name)
        pr.close()


def test_device_plan_is_the_exchange_layout(cuda_lib):
    g = load_golden("beem_medium.json")
    m = synth.beem_shaped_model(**g["model"])
    pr = cuda_lib.PartReach(4, 22, m.state_words, exchange_rows=1 << 16)
    got, _, _ = pr.run(m)
    assert got.states == g["states"] and got.digest == int(g["digest"], 16)
    counts, seg, begin = pr.last_exchange()
    want_seg, want_begin = exchange.plan(counts)
    assert counts.sum() > 0
    assert np.array_equal(seg.astype(np.int64), want_seg)
    assert np.array_equal(begin.astype(np.int64), want_begin)
    pr.close()


def test_overflowing_partition_is_reported(cuda_lib):
    m = synth.sized_interleaving_model(7, 4, 16, 40000)   # 40k states into 2 x 2^10 buckets
    pr = cuda_lib.PartReach(2, 10, m.state_words)
    got, _, _ = pr.run(m, raise_on_error=False)
    assert got.status == cuda_lib.HT_ERR_FULL
    # the same object runs a model that fits afterwards (every table is cleared)
    small = synth.sized_interleaving_model(3, 3, 16, 500)
    got, parts, _ = pr.run(small)
    _same(got, oracle.reach(small))
    pr.close()


def test_invalid_shapes_are_refused(cuda_lib):
    for K, lg, W, rows in ((3, 12, 16, 1 << 16), (32, 12, 16, 1 << 16), (2, 9, 16, 1 << 16),
                           (2, 12, 33, 1 << 16), (2, 12, 16, 100)):
        with pytest.raises(cuda_lib.HtError):
            cuda_lib.part_reach_bytes(K, lg, W, rows)
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.PartReach(2, 12, 16, bucket_bits=16)
