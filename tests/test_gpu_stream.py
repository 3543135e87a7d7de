"""Device key streams and fused find-or-put against the host generator and the oracle.

The device generator must produce exactly the keys of the seeded input
generator (byte-exact), and find-or-put over a generated fill must store
exactly the fill's distinct keys (count and set digest equal to the oracle's
on the host-generated keys).
"""
import numpy as np
import pytest

import oracle
from paper_1004_2772_gb300 import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("W", [1, 5, 16, 32])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_device_keys_equal_host_keys(cuda_lib, W, dist):
    n_ids = 5000
    zt = synth.zipf_table(n_ids) if dist == "zipf" else None
    tab = cuda_lib.Table(8, W)
    for c0, n in [(0, 2 * n_ids), (777, 1234)]:
        dev = tab.gen_keys(31, n_ids, c0, n, zt).cpu().numpy()
        host = synth.key_words(31, synth.call_ids(31, n_ids, c0, n, dist, zt), W)
        assert np.array_equal(dev, host)


@pytest.mark.parametrize("L", [8, 16, 32])
@pytest.mark.parametrize("dedup", [0, 1])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_fused_stream_matches_oracle(cuda_lib, L, dedup, dist):
    n_ids = 1 << 14
    zt = synth.zipf_table(n_ids) if dist == "zipf" else None
    ids = synth.call_ids(9, n_ids, 0, 2 * n_ids, dist, zt)
    ref = oracle.find_or_put_stream(synth.key_words(9, ids, 16))
    tab = cuda_lib.Table(16, 16, line_buckets=L, dedup=dedup)
    tot_new, tot_dig = 0, 0
    for c0, n in [(0, 10000), (10000, 2 * n_ids - 10000)]:   # two calls, like two batches
        k, d = tab.find_or_put_stream(9, n_ids, c0, n, zt)
        tot_new += k
        tot_dig = (tot_dig + d) % (1 << 64)
    assert (tot_new, tot_dig) == (ref.n_new, ref.digest) == (n_ids, ref.digest)
    done, writing, digest = tab.scan()
    assert (done, writing, digest) == (n_ids, 0, ref.digest)
    assert tab.sync() == cuda_lib.HT_OK


def test_batch_api_and_fused_agree(cuda_lib):
    torch = _torch()
    n_ids = 1 << 15
    a = cuda_lib.Table(17, 16)
    b = cuda_lib.Table(17, 16)
    keys = a.gen_keys(4, n_ids, 0, 2 * n_ids)
    seen, idx = a.find_or_put(keys)
    torch.cuda.synchronize()
    n_new, dig = b.find_or_put_stream(4, n_ids, 0, 2 * n_ids)
    assert int((seen == 0).sum()) == n_new == n_ids
    assert a.scan() == b.scan()


def test_fused_stream_at_scale_properties(cuda_lib):
    """2^24 buckets at load factor 0.9 (15.1M keys, 30.2M calls): every id is
    stored exactly once, whatever the interleaving; the digest of the fill is
    the oracle's digest of the distinct keys, computed in chunks."""
    log2 = 24
    n_ids = int(0.9 * (1 << log2))
    tab = cuda_lib.Table(log2, 16, line_buckets=32)
    n_new, dig = tab.find_or_put_stream(77, n_ids, 0, 2 * n_ids)
    assert n_new == n_ids
    want = 0
    for lo in range(0, n_ids, 1 << 21):
        ids = np.arange(lo, min(n_ids, lo + (1 << 21)), dtype=np.uint64)
        want = (want + oracle.digest(synth.key_words(77, ids, 16))) % (1 << 64)
    assert dig == want
    done, writing, digest = tab.scan()
    assert (done, writing, digest) == (n_ids, 0, want)
