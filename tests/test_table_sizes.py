"""Tables whose size is not a power of two (Section 3.1: constant division).

Host side (no GPU): the library's invariant-divisor division gives exactly
n // d and n % d (Granlund-Montgomery guarantee it for every 64-bit n; checked
here at the edges and on random values), and the sizing helpers return the
largest fitting table with a prime line count.  GPU side: parity of
non-power-of-two tables against the oracle, through the C ABI.
"""
import numpy as np
import pytest

import oracle
from conftest import hand_models, load_golden
from paper_1004_2772_gb300 import binding, synth

U64 = (1 << 64) - 1


def _is_prime(n):
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    f = 3
    while f * f <= n:
        if n % f == 0:
            return False
        f += 2
    return True


def _divisors():
    ds = {1, 2, 3, 5, 7, 8, 9, 10, 641, 6700417, (1 << 31) - 1, (1 << 32) - 1, (1 << 32) - 5}
    for k in range(1, 32):
        ds |= {(1 << k) - 1, 1 << k, (1 << k) + 1}
    rng = np.random.default_rng(5)
    ds |= {int(x) for x in rng.integers(1, 1 << 32, size=60, dtype=np.uint64)}
    ds |= {int(x) for x in rng.integers(1, 1 << 12, size=30, dtype=np.uint64)}
    return sorted(d for d in ds if 1 <= d < (1 << 32))


def _dividends(d, rng):
    vals = {0, 1, 2, U64, U64 - 1, 1 << 63, (1 << 63) - 1, (1 << 32) - 1, 1 << 32}
    for m in (1, 2, 3, U64 // d - 1, U64 // d):
        for e in (-1, 0, 1):
            v = m * d + e
            if 0 <= v <= U64:
                vals.add(v)
    vals |= {int(x) for x in rng.integers(0, 1 << 63, size=200, dtype=np.uint64) * 2 + 1}
    return np.array(sorted(vals), dtype=np.uint64)


def test_line_division_is_exact():
    rng = np.random.default_rng(11)
    for d in _divisors():
        n = _dividends(d, rng)
        q, r = binding.vss_line_divide(d, n)
        for a, qa, ra in zip(n.tolist(), q.tolist(), r.tolist()):
            assert (qa, ra) == divmod(a, d), (d, a)


def test_line_division_rejects_zero():
    with pytest.raises(binding.HtError):
        binding.vss_line_divide(0, np.zeros(1, dtype=np.uint64))


@pytest.mark.parametrize("L", [8, 16, 32])
@pytest.mark.parametrize("W", [1, 5, 16, 32])
def test_buckets_for_bytes_is_largest_prime_line_table(L, W):
    p = binding.make_params(line_buckets=L)
    for budget in (1 << 20, 3 << 24, 10_000_000_000 // 7):
        nb = binding.ht_buckets_for_bytes(budget, W, p)
        assert nb % L == 0 and binding.ht_bytes_n(nb, W) <= budget
        lines = nb // L
        assert _is_prime(lines) or lines & (lines - 1) == 0
        nxt = lines + 1
        while not _is_prime(nxt):
            nxt += 1
        big = nxt * L
        assert big > (1 << 31) or binding.ht_bytes_n(big, W) > budget


def test_reach_ctx_buckets_for_bytes_fits():
    budget = 5 << 30
    nb = binding.reach_ctx_buckets_for_bytes(budget, 16, 4096)
    assert _is_prime(nb // 32) and binding.reach_ctx_bytes_n(nb, 16, 4096) <= budget   # default 32-bucket lines
    assert binding.reach_ctx_bytes_n(nb, 16, 4096) > 0.95 * budget


def test_invalid_sizes_rejected():
    with pytest.raises(binding.HtError):
        binding.ht_bytes_n(8, 16)                     # below the minimum
    with pytest.raises(binding.HtError):
        binding.ht_bytes_n((1 << 31) + 8, 16)         # above 2^31
    with pytest.raises(binding.HtError):
        binding.ht_buckets_for_bytes(100, 16)          # nothing fits


# ---------------------------------------------------------------------------
# GPU parity
# ---------------------------------------------------------------------------

def _prime_lines_near(n_lines):
    while not _is_prime(n_lines):
        n_lines -= 1
    return n_lines


@pytest.mark.gpu
@pytest.mark.parametrize("W", [1, 5, 16, 32])
@pytest.mark.parametrize("layout", [(32, 8), (32, 32), (16, 16)])
def test_stream_parity_non_pow2(cuda_lib, W, layout):
    from test_gpu_table import check_parity, run_batches
    bw, L = layout
    nb = _prime_lines_near(60000 // L) * L
    n_ids = 20000
    ids = synth.call_ids(W + L + 3, n_ids, 0, 2 * n_ids, "uniform")
    keys = synth.key_words(W * 11 + L, ids, W)
    keys = np.ascontiguousarray(keys[np.random.default_rng(W).permutation(keys.shape[0])])
    tab = cuda_lib.Table(None, W, n_buckets=nb, line_buckets=L, bucket_bits=bw)
    assert tab.stats().capacity == nb
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 3)
    assert int(idx.max()) < nb
    check_parity(tab, keys, seen, idx, cuts)


@pytest.mark.gpu
@pytest.mark.parametrize("lines", [3, 5, 97, 1009, 7919])
def test_high_load_non_pow2(cuda_lib, lines):
    """95% load: long walks and rehashes over a prime line count."""
    from test_gpu_table import check_parity, run_batches
    nb = lines * 8
    n_ids = int(0.95 * nb)
    ids = np.repeat(np.arange(n_ids, dtype=np.uint64), 2)
    np.random.default_rng(lines).shuffle(ids)
    keys = synth.key_words(lines, ids, 16)
    tab = cuda_lib.Table(None, 16, n_buckets=nb, line_buckets=8)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 1)
    check_parity(tab, keys, seen, idx, cuts)


@pytest.mark.gpu
def test_full_non_pow2_table_reports_full(cuda_lib):
    import torch
    keys = synth.key_words(9, np.arange(60, dtype=np.uint64), 16)
    tab = cuda_lib.Table(None, 16, n_buckets=5 * 8, line_buckets=8)     # 5 lines of 8
    s, _ = tab.find_or_put(torch.from_numpy(keys).cuda())
    torch.cuda.synchronize()
    s = s.cpu().numpy()
    assert tab.sync() == cuda_lib.HT_ERR_FULL
    done, writing, _ = tab.scan()
    assert writing == 0 and done == (s == 0).sum() == 40   # every bucket of a prime-line table is reachable


@pytest.mark.gpu
def test_fused_stream_non_pow2(cuda_lib):
    n_ids = 1 << 14
    ids = synth.call_ids(9, n_ids, 0, 2 * n_ids, "uniform")
    ref = oracle.find_or_put_stream(synth.key_words(9, ids, 16))
    tab = cuda_lib.Table(None, 16, n_buckets=_prime_lines_near(40000 // 32) * 32)  # default line
    n_new, dig = tab.find_or_put_stream(9, n_ids, 0, 2 * n_ids)
    assert (n_new, dig) == (ref.n_new, ref.digest)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_reach_non_pow2(cuda_lib, mode):
    from test_gpu_reach import check
    m = synth.tiny_interleaving_model()
    ctx = cuda_lib.ReachContext(None, 5, max_levels=256, n_buckets=_prime_lines_near(150000 // 32) * 32)
    got = check(cuda_lib, ctx, m, mode)
    assert got.states == 100000
    ctx2 = cuda_lib.ReachContext(None, 8, max_levels=64, n_buckets=13 * 8, line_buckets=8)
    for hm, d in hand_models():
        check(cuda_lib, ctx2, hm, mode)


@pytest.mark.gpu
def test_beem_shaped_medium_non_pow2(cuda_lib):
    g = load_golden("beem_medium.json")
    m = synth.beem_shaped_model(**g["model"])
    nb = _prime_lines_near(int(1.5 * g["states"]) // 32) * 32        # load factor ~0.67
    ctx = cuda_lib.ReachContext(None, 16, max_levels=4096, n_buckets=nb)
    for mode in (0, 1, 2):
        got = ctx.reach(m, mode=mode)
        assert (got.states, got.transitions, got.deadlocks, got.digest) == (
            g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
        assert got.level_sizes == g["level_sizes"]
        done, writing, digest = ctx.scan()
        assert (done, writing, digest) == (g["states"], 0, int(g["digest"], 16))


@pytest.mark.gpu
def test_beem_shaped_workload_full_size_non_pow2(cuda_lib):
    """The 32M-state workload in the largest prime-line context that fits a
    12 GiB budget, against the oracle's stored result."""
    g = load_golden("beem_c2.json")
    m = synth.beem_shaped_model(**g["model"])
    nb = cuda_lib.reach_ctx_buckets_for_bytes(12 << 30, 16, 1 << 14)
    assert nb & (nb - 1) != 0 and nb > g["states"]
    ctx = cuda_lib.ReachContext(None, 16, max_levels=1 << 14, n_buckets=nb)
    got = ctx.reach(m, mode=0)
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
    assert got.level_sizes == g["level_sizes"]
