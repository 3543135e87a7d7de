"""reach_noalloc, the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- e.g. a process whose device memory is
fixed when it starts -- so reach_noalloc runs the persistent reachability
driver out of a fixed 32 MiB array that the library itself holds on the GPU.
This file checks, through the C ABI, that it gives the CPU oracle's answer
(states, transitions, deadlocks, level sizes and set digest, bit-exact) and
the same answer as the context-based reach(), on two calls in a row (the
array keeps the previous call's contents, so the second call also checks that
everything is cleared), and that requests larger than the array are refused.
It is collected last so that a failure here cannot hide any other test, and
it passes both alone in a fresh process and after the rest of the suite.
"""
import pytest

import oracle
from paper_1004_2772_gb300 import synth

pytestmark = pytest.mark.gpu


def _same(a_st, a, a_levels, ref):
    assert a_st == 0
    assert (a.states, a.transitions, a.deadlocks, a.digest) == (
        ref.states, ref.transitions, ref.deadlocks, ref.digest)
    assert [int(x) for x in a_levels] == ref.level_sizes


CASES = [
    (synth.tiny_interleaving_model(), 18),                       # W = 5, 10^5 states
    (synth.beem_shaped_model(3, n_procs=8, n_shared=3, state_words=16, n_lo=3, n_hi=5,
                             update_pct=40), 17),                 # W = 16, guarded
]


@pytest.mark.parametrize("case", CASES, ids=["tiny-W5", "guarded-W16"])
def test_no_alloc_matches_oracle_and_reach_twice(cuda_lib, case):
    b = cuda_lib
    m, log2 = case
    ref = oracle.reach(m)
    assert not ref.truncated
    ctx = b.ReachContext(log2, m.state_words, max_levels=4096)
    alone = ctx.reach(m)
    ctx.close()
    _same(0, alone, alone.level_sizes, ref)
    for _ in range(2):
        st, r, levels = b.reach_noalloc(m, log2, max_levels=4096)
        _same(st, r, levels, ref)


def test_no_alloc_refuses_oversized_requests(cuda_lib):
    b = cuda_lib
    m = synth.tiny_interleaving_model()
    st, r, _ = b.reach_noalloc(m, 24, max_levels=4096)   # 2^24 buckets: far beyond 32 MiB
    assert st == b.HT_ERR_TOO_BIG
    st, r, levels = b.reach_noalloc(m, 18, max_levels=4096)  # still usable afterwards
    _same(st, r, levels, oracle.reach(m))


def test_no_alloc_16_bit_buckets(cuda_lib):
    b = cuda_lib
    m = synth.tiny_interleaving_model()
    ref = oracle.reach(m)
    st, r, levels = b.reach_noalloc(m, 18, b.make_params(bucket_bits=16), max_levels=4096)
    _same(st, r, levels, ref)


@pytest.mark.parametrize("G", [2, 8])
def test_no_alloc_with_lane_groups(cuda_lib, G):
    """Cooperative probing (groups of G lanes, lines of 4G buckets) through
    the fixed array too."""
    b = cuda_lib
    m = synth.tiny_interleaving_model()
    ref = oracle.reach(m)
    st, r, levels = b.reach_noalloc(m, 18, b.make_params(group_lanes=G, line_buckets=4 * G),
                                    max_levels=4096)
    _same(st, r, levels, ref)
