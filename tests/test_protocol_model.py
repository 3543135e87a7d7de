"""Protocol-as-model check: the find-or-put protocol explored by reach().

Every interleaving of T threads inserting keys into a line of B buckets is a
reachable state of the protocol model (tests/protocol_model.py).  The oracle
enumerates them and every reachable state is checked: no key is ever stored
twice, and when every thread has finished exactly one of the threads inserting
a key was told "new".  A planted version of the write-bit mistake must break
this.  The GPU reach() must produce the same state space (-m gpu).
"""
import pytest

import oracle
from protocol_model import protocol_model, violations

CASES = [
    # (keys, memos, buckets): equal keys race for one bucket; keys sharing a memo force
    # the data compare; more threads than buckets exercise the walk to the next bucket
    ((1, 1), (1, 1), 2),
    ((1, 1, 1), (1, 1, 1), 2),
    ((1, 2), (1, 1), 2),
    ((1, 2, 1), (1, 1, 1), 3),
    ((1, 2, 3), (1, 2, 1), 3),
    ((1, 1, 2, 2), (1, 1, 1, 1), 2),
]


@pytest.mark.parametrize("case", CASES, ids=[f"T{len(c[0])}-B{c[2]}-{i}" for i, c in enumerate(CASES)])
def test_protocol_has_no_duplicates_and_one_new_per_key(case):
    keys, memos, B = case
    m = protocol_model(keys, memos, B)
    r = oracle.reach(m, keep_states=True, max_states=2_000_000)
    assert not r.truncated and r.states > 1
    assert violations(m, r.state_list) == []
    assert r.deadlocks > 0          # the terminal states: every thread finished


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3]])
def test_planted_write_bit_mistake_is_found(case):
    keys, memos, B = case
    m = protocol_model(keys, memos, B, broken="skip_write")
    r = oracle.reach(m, keep_states=True, max_states=2_000_000)
    bad = violations(m, r.state_list)
    assert any(v[0] == "duplicate" for v in bad)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[f"T{len(c[0])}-B{c[2]}-{i}" for i, c in enumerate(CASES)])
def test_gpu_reach_explores_the_same_protocol_space(cuda_lib, case):
    keys, memos, B = case
    for broken in (None, "skip_write"):
        m = protocol_model(keys, memos, B, broken=broken)
        ref = oracle.reach(m)
        ctx = cuda_lib.ReachContext(14, m.state_words, max_levels=4096)
        got = ctx.reach(m)
        assert (got.states, got.transitions, got.deadlocks, got.digest, got.level_sizes) == (
            ref.states, ref.transitions, ref.deadlocks, ref.digest, ref.level_sizes)
        ctx.close()
