"""The rehash rule (ht_params.rehash): after a full line, the next line by
double hashing (default) or simply the next line.  Both probe sequences are
deterministic and never re-empty a bucket, so both must store exactly the
oracle's set; at high load the walks really do leave their first line.
"""
import numpy as np
import pytest

import oracle
from conftest import load_golden
from paper_1004_2772_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rehash", [0, 1])
@pytest.mark.parametrize("L", [8, 32])
def test_high_load_fill_matches_oracle(cuda_lib, rehash, L):
    log2 = 14
    n_ids = int(0.97 * (1 << log2))
    ids = synth.call_ids(5, n_ids, 0, 2 * n_ids)
    ref = oracle.find_or_put_stream(synth.key_words(5, ids, 16))
    tab = cuda_lib.Table(log2, 16, line_buckets=L, rehash=rehash)
    n_new, dig = tab.find_or_put_stream(5, n_ids, 0, 2 * n_ids)
    assert (n_new, dig) == (ref.n_new, ref.digest)
    assert tab.scan() == (n_ids, 0, ref.digest)
    st = tab.stats()
    assert st.rehashes > 0 and st.error == 0


def test_prime_line_table_next_line(cuda_lib):
    """A table of any size (prime line count) with the next-line rule."""
    n_ids = 9000
    ids = synth.call_ids(6, n_ids, 0, 2 * n_ids)
    ref = oracle.find_or_put_stream(synth.key_words(6, ids, 16))
    nb = 32 * 313
    tab = cuda_lib.Table(None, 16, n_buckets=nb, rehash=1)
    n_new, dig = tab.find_or_put_stream(6, n_ids, 0, 2 * n_ids)
    assert (n_new, dig) == (n_ids, ref.digest)


@pytest.mark.parametrize("rehash", [0, 1])
def test_reach_with_either_rule(cuda_lib, rehash):
    g = load_golden("beem_medium.json")
    m = synth.beem_shaped_model(**g["model"])
    ctx = cuda_lib.ReachContext(23, m.state_words, rehash=rehash)   # load 0.65
    got = ctx.reach(m)
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
    assert got.level_sizes == g["level_sizes"]
    ctx.close()


def test_batch_and_serving_refuse_the_next_line_rule(cuda_lib):
    models = synth.batched_models(count=2, first_seed=1)
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.ReachBatch(models, rehash=1)
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.Server(budget_bytes=1 << 28, n_slots=2, rehash=1)
