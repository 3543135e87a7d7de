"""Sub-warp cooperative find-or-put (ht_params.group_lanes = 2, 4, 8) against
the oracle: G lanes read a whole line of 4G buckets at once and must reach the
same sets, counts and per-key properties as one thread walking the line."""
import numpy as np
import pytest

import oracle
from paper_1004_2772_gb300 import synth
from test_gpu_table import check_parity, run_batches

pytestmark = pytest.mark.gpu

GROUPS = [2, 4, 8]


@pytest.mark.parametrize("W", [1, 5, 16, 32])
@pytest.mark.parametrize("G", GROUPS)
def test_stream_parity_shapes(cuda_lib, W, G):
    n_ids = 20000
    ids = synth.call_ids(W + 7 * G, n_ids, 0, 2 * n_ids, "uniform")
    keys = synth.key_words(W * 13 + G, ids, W)
    keys = np.ascontiguousarray(keys[np.random.default_rng(W + G).permutation(keys.shape[0])])
    tab = cuda_lib.Table(16, W, group_lanes=G)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 3)
    check_parity(tab, keys, seen, idx, cuts)
    assert tab.sync() == cuda_lib.HT_OK


@pytest.mark.parametrize("dist", ["uniform", "zipf"])
@pytest.mark.parametrize("G", GROUPS)
def test_stream_parity_hot_keys(cuda_lib, dist, G):
    n_ids = 1 << 15
    zt = synth.zipf_table(n_ids) if dist == "zipf" else None
    ids = synth.call_ids(81, n_ids, 0, 2 * n_ids, dist, zt)
    keys = synth.key_words(82, ids, 16)
    tab = cuda_lib.Table(16, 16, group_lanes=G)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 4)
    check_parity(tab, keys, seen, idx, cuts)


@pytest.mark.parametrize("G", GROUPS)
@pytest.mark.parametrize("size", [("pow2", 1 << 10), ("prime-lines", None)])
def test_high_load_forces_rehash(cuda_lib, G, size):
    kind, nb = size
    if nb is None:
        nb = 4 * G * 251                            # 251 lines (prime)
    n_ids = int(0.95 * nb)
    ids = np.repeat(np.arange(n_ids, dtype=np.uint64), 3)
    np.random.default_rng(G).shuffle(ids)
    keys = synth.key_words(7, ids, 16)
    tab = cuda_lib.Table(None, 16, n_buckets=nb, group_lanes=G)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 1)
    check_parity(tab, keys, seen, idx, cuts)
    assert tab.stats().rehashes > 0


@pytest.mark.parametrize("G", GROUPS)
def test_full_table_reports_full(cuda_lib, G):
    import torch
    keys = synth.key_words(9, np.arange(3 * 32, dtype=np.uint64), 16)
    tab = cuda_lib.Table(5, 16, group_lanes=G)     # 32 buckets
    s, _ = tab.find_or_put(torch.from_numpy(keys).cuda())
    torch.cuda.synchronize()
    s = s.cpu().numpy()
    assert tab.sync() == cuda_lib.HT_ERR_FULL
    done, writing, _ = tab.scan()
    assert writing == 0 and done == (s == 0).sum() == 32


@pytest.mark.parametrize("dist", ["uniform", "zipf"])
@pytest.mark.parametrize("G", GROUPS)
def test_fused_stream_matches_oracle(cuda_lib, dist, G):
    n_ids = 1 << 14
    zt = synth.zipf_table(n_ids) if dist == "zipf" else None
    ids = synth.call_ids(12, n_ids, 0, 2 * n_ids, dist, zt)
    ref = oracle.find_or_put_stream(synth.key_words(12, ids, 16))
    tab = cuda_lib.Table(16, 16, group_lanes=G)
    n_new, dig = tab.find_or_put_stream(12, n_ids, 0, 2 * n_ids, zt)
    assert (n_new, dig) == (ref.n_new, ref.digest)
    assert tab.scan() == (n_ids, 0, ref.digest)


def test_group_parameters_validated(cuda_lib):
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.Table(10, 4, group_lanes=3)
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.Table(10, 4, group_lanes=4, line_buckets=8)
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.Table(10, 4, group_lanes=4, bucket_bits=16)
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.ReachContext(10, 4, group_lanes=4, line_buckets=32)
    # tracing is compiled for one lane per successor only
    ctx = cuda_lib.ReachContext(18, 5, group_lanes=4)
    got = ctx.reach(synth.tiny_interleaving_model(), mode=cuda_lib.REACH_PERSISTENT | cuda_lib.REACH_TRACE,
                    raise_on_error=False)
    assert got.status == cuda_lib.HT_ERR_INVALID
    # the many-model kernels take one lane per key
    with pytest.raises(cuda_lib.HtError):
        cuda_lib.ReachBatch([synth.tiny_interleaving_model()], group_lanes=4)


# ---------------------------------------------------------------------------
# Reachability with cooperative probing: the G lanes of a group build the same
# successor and walk its line of 4G buckets together.
# ---------------------------------------------------------------------------

def _reach_check(cuda_lib, ctx, m, mode, ref):
    from test_gpu_reach import check
    return check(cuda_lib, ctx, m, mode, ref)


@pytest.mark.parametrize("G", GROUPS)
def test_reach_with_groups_tiny_and_guarded(cuda_lib, G):
    """The tiny interleaving model (rows of 5 words) and guarded models with
    rows of 13, 16 and 32 words, in all three drivers."""
    from test_gpu_reach import MODES, log2_for
    cases = [(synth.tiny_interleaving_model(), 18)]
    for W in (13, 16, 32):
        cases.append((synth.beem_shaped_model(13, n_procs=10, n_shared=3, state_words=W, n_lo=3, n_hi=6,
                                              update_pct=40), None))
    for m, lg in cases:
        ref = oracle.reach(m)
        ctx = cuda_lib.ReachContext(lg or log2_for(ref.states), m.state_words, max_levels=4096,
                                    group_lanes=G)
        for mode in MODES:
            _reach_check(cuda_lib, ctx, m, mode, ref)
        ctx.close()


@pytest.mark.parametrize("G", GROUPS)
def test_reach_with_groups_high_load_prime_lines(cuda_lib, G):
    """A table of a prime number of lines at load 0.9: walks rehash."""
    m = synth.beem_shaped_model(13, n_procs=10, n_shared=3, state_words=16, n_lo=3, n_hi=6, update_pct=40)
    ref = oracle.reach(m)
    lines = {8: 2113, 4: 4229, 2: 8461}[G]                      # primes: load 0.90 with 4G-bucket lines
    ctx = cuda_lib.ReachContext(None, 16, n_buckets=4 * G * lines, max_levels=4096, group_lanes=G)
    got = _reach_check(cuda_lib, ctx, m, 0, ref)
    assert got.rehashes > 0
    ctx.close()


@pytest.mark.parametrize("G", [4, 8])
def test_reach_with_groups_medium_golden(cuda_lib, G):
    """The 5.5M-state BEEM-shaped medium model against its stored values."""
    from conftest import load_golden
    g = load_golden("beem_medium.json")
    m = synth.beem_shaped_model(seed=7, update_pct=40)
    ctx = cuda_lib.ReachContext(24, 16, max_levels=4096, group_lanes=G)
    r = ctx.reach(m)
    assert (r.states, r.transitions, r.deadlocks, r.digest, r.level_sizes) == (
        g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16), g["level_sizes"])
    done, writing, digest = ctx.scan()
    assert (done, writing, digest) == (g["states"], 0, r.digest)
    ctx.close()
