"""The 16-bit bucket layout (ht_params.bucket_bits = 16) against the oracle.

Same bars as the 32-bit tests: bit-exact sets, counts, level sizes and
digests; per-key properties for the batch API.  A 15-bit memo lets about one
foreign key in 2^15 through to a data compare, so the high-load cases also
exercise the memo-equal / data-unequal branch of the walk.
"""
import numpy as np
import pytest

import oracle
from conftest import hand_models, load_golden
from paper_1004_2772_gb300 import synth
from test_gpu_reach import MODES, check
from test_gpu_table import check_parity, run_batches
from test_oracle_pins import TINY_BEEM

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W", [1, 5, 16, 32])
@pytest.mark.parametrize("L", [16, 32])
def test_stream_parity_shapes(cuda_lib, W, L):
    rng = np.random.default_rng(W * 100 + L + 1)
    n_ids = 20000
    ids = synth.call_ids(W + L + 1, n_ids, 0, 2 * n_ids, "uniform")
    keys = synth.key_words(W * 7 + L + 1, ids, W)
    keys = np.ascontiguousarray(keys[rng.permutation(keys.shape[0])])
    tab = cuda_lib.Table(16, W, line_buckets=L, bucket_bits=16)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 3)
    check_parity(tab, keys, seen, idx, cuts)
    assert tab.sync() == cuda_lib.HT_OK


@pytest.mark.parametrize("dedup", [0, 1])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_stream_parity_hot_keys(cuda_lib, dedup, dist):
    n_ids = 1 << 15
    zt = synth.zipf_table(n_ids) if dist == "zipf" else None
    ids = synth.call_ids(79, n_ids, 0, 2 * n_ids, dist, zt)
    keys = synth.key_words(80, ids, 16)
    tab = cuda_lib.Table(16, 16, dedup=dedup, bucket_bits=16)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 4)
    check_parity(tab, keys, seen, idx, cuts)


@pytest.mark.parametrize("lf_log2", [(6, 60), (8, 240), (12, 4000), (16, 63000)])
def test_high_load_forces_rehash(cuda_lib, lf_log2):
    log2, n_ids = lf_log2
    ids = np.repeat(np.arange(n_ids, dtype=np.uint64), 3)
    np.random.default_rng(log2 + 1).shuffle(ids)
    keys = synth.key_words(6, ids, 16)
    tab = cuda_lib.Table(log2, 16, bucket_bits=16)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 1)
    check_parity(tab, keys, seen, idx, cuts)
    assert tab.stats().rehashes > 0


def test_full_table_reports_full(cuda_lib):
    import torch
    keys = synth.key_words(9, np.arange(40, dtype=np.uint64), 16)
    tab = cuda_lib.Table(4, 16, bucket_bits=16)   # 16 buckets = one line
    s, _ = tab.find_or_put(torch.from_numpy(keys).cuda())
    torch.cuda.synchronize()
    s = s.cpu().numpy()
    assert tab.sync() == cuda_lib.HT_ERR_FULL
    done, writing, _ = tab.scan()
    assert writing == 0 and done == (s == 0).sum() == 16


def test_bucket_words_have_the_16_bit_layout(cuda_lib):
    n_ids = 5000
    keys = synth.key_words(11, np.arange(n_ids, dtype=np.uint64), 8)
    tab = cuda_lib.Table(14, 8, bucket_bits=16)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 2)
    b, data = tab.arrays()
    w = b.cpu().numpy().view(np.uint16)
    used = np.nonzero(w)[0]
    assert used.shape[0] == n_ids
    assert (w[used] & 0x8000).all()                       # every used bucket is done
    assert ((w[used] & 0x7FFF) != 0).all()               # memo never 0
    assert np.array_equal(np.sort(used), np.sort(idx))    # keys live where their buckets are
    assert np.array_equal(data.cpu().numpy()[idx], keys)


def test_invalid_width_and_line(cuda_lib):
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.Table(10, 4, bucket_bits=16, line_buckets=8)
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.Table(10, 4, bucket_bits=24)
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.ReachBatch([synth.tiny_interleaving_model()], log2_initial=[10], bucket_bits=16)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L", [16, 32])
def test_tiny_interleaving(cuda_lib, mode, L):
    m = synth.tiny_interleaving_model()
    ctx = cuda_lib.ReachContext(18, 5, max_levels=256, line_buckets=L, bucket_bits=16)
    got = check(cuda_lib, ctx, m, mode)
    assert got.states == 100000 and got.transitions == 1000000


@pytest.mark.parametrize("mode", MODES)
def test_hand_models(cuda_lib, mode):
    ctx = cuda_lib.ReachContext(8, 8, max_levels=64, bucket_bits=16)
    for m, d in hand_models():
        got = check(cuda_lib, ctx, m, mode)
        assert got.states == d["states"] and got.level_sizes == d["level_sizes"]


@pytest.mark.parametrize("kw", TINY_BEEM, ids=[f"seed{k['seed']}" for k in TINY_BEEM])
def test_tiny_guarded_models(cuda_lib, kw):
    m = synth.beem_shaped_model(**kw)
    ctx = cuda_lib.ReachContext(12, m.state_words, max_levels=1024, bucket_bits=16)
    for mode in MODES:
        check(cuda_lib, ctx, m, mode)


def test_beem_shaped_medium(cuda_lib):
    g = load_golden("beem_medium.json")
    m = synth.beem_shaped_model(**g["model"])
    ctx = cuda_lib.ReachContext(g["log2_buckets"], 16, max_levels=4096, bucket_bits=16)
    for mode in MODES:
        got = ctx.reach(m, mode=mode)
        assert (got.states, got.transitions, got.deadlocks, got.digest) == (
            g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
        assert got.level_sizes == g["level_sizes"]


def test_beem_shaped_workload_full_size(cuda_lib):
    """The benchmarked BEEM-shaped workload (32M states, 2^26 buckets) on a
    16-bit bucket table, against the oracle's stored result."""
    g = load_golden("beem_c2.json")
    m = synth.beem_shaped_model(**g["model"])
    ctx = cuda_lib.ReachContext(g["log2_buckets"], 16, max_levels=1 << 14, bucket_bits=16)
    got = ctx.reach(m, mode=0)
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
    assert got.level_sizes == g["level_sizes"]
    done, writing, digest = ctx.scan()
    assert (done, writing, digest) == (g["states"], 0, int(g["digest"], 16))


def test_deadlock_trace(cuda_lib):
    kws = [kw for kw in TINY_BEEM if oracle.reach(synth.beem_shaped_model(**kw)).deadlocks > 0]
    m = synth.beem_shaped_model(**kws[0])
    ref = oracle.reach(m)
    ctx = cuda_lib.ReachContext(12, m.state_words, max_levels=4096, bucket_bits=16)
    got = ctx.reach(m, mode=cuda_lib.REACH_PERSISTENT | cuda_lib.REACH_TRACE)
    assert (got.states, got.deadlocks, got.digest) == (ref.states, ref.deadlocks, ref.digest)
    level, path = ctx.deadlock_trace()
    from test_gpu_reach import _check_trace
    _check_trace(m, level, path, ref)

