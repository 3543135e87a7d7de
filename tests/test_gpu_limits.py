"""The largest table the C ABI allows (2^31 buckets) on the GPU's own memory.

With W = 16 a 2^31-bucket table takes 146 GB; the test runs only when the
device has that much free.  Bucket indices then use all 31 bits, row offsets
pass 2^37 bytes, and the scan walks 8 GiB of buckets: a fill of 2^24 distinct
keys (2^25 calls) must store exactly the distinct keys and their oracle
digest, and a prime-line table just below the limit must do the same; a
reachability context of 200 GB must reproduce the 32M-state workload.
"""
import numpy as np
import pytest

import oracle
from paper_1004_2772_gb300 import synth

pytestmark = pytest.mark.gpu


def _oracle_digest(seed, n_ids):
    want = 0
    for lo in range(0, n_ids, 1 << 21):
        ids = np.arange(lo, min(n_ids, lo + (1 << 21)), dtype=np.uint64)
        want = (want + oracle.digest(synth.key_words(seed, ids, 16))) % (1 << 64)
    return want


def _need_free(nbytes):
    import gc

    import torch
    # memory that earlier tests' tensors left in torch's cache goes back to the driver first
    gc.collect()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < nbytes + (8 << 30):
        pytest.skip(f"needs {nbytes / 1e9:.0f} GB free on the device, {free / 1e9:.0f} GB free")


@pytest.mark.parametrize("kind", ["pow2", "prime-lines"])
def test_largest_table(cuda_lib, kind):
    import torch
    if kind == "pow2":
        kw = dict(log2_buckets=31)
        nbytes = cuda_lib.ht_bytes(31, 16)
    else:
        nb = cuda_lib.ht_buckets_for_bytes(cuda_lib.ht_bytes(31, 16) - (1 << 30), 16)
        assert nb & (nb - 1) != 0 and nb > (1 << 30)
        kw = dict(log2_buckets=None, n_buckets=nb)
        nbytes = cuda_lib.ht_bytes_n(nb, 16)
    _need_free(nbytes)
    tab = cuda_lib.Table(kw.pop("log2_buckets"), 16, **kw)
    n_ids = 1 << 24
    n_new, dig = tab.find_or_put_stream(91, n_ids, 0, 2 * n_ids)
    assert n_new == n_ids
    assert dig == _oracle_digest(91, n_ids)
    done, writing, digest = tab.scan()
    assert (done, writing, digest) == (n_ids, 0, dig)
    # the batch API on the same table: every key is now seen, at its bucket
    keys = tab.gen_keys(91, n_ids, 0, 1 << 16)
    seen, idx = tab.find_or_put(keys)
    torch.cuda.synchronize()
    assert bool((seen == 1).all())
    got = tab.gather(idx)
    assert torch.equal(got, keys)
    st = tab.stats()
    assert st.error == 0 and st.capacity == tab.n_buckets
    tab.close()
    del tab
    torch.cuda.empty_cache()


def test_largest_reach_context(cuda_lib):
    """The 32M-state BEEM-shaped workload in the largest prime-line context
    that fits 200 GB (about 8.7e8 buckets: frontiers of that many rows),
    against the oracle's stored result."""
    import torch
    from conftest import load_golden
    budget = 200 << 30
    _need_free(budget)
    nb = cuda_lib.reach_ctx_buckets_for_bytes(budget, 16, 1 << 14)
    assert nb > (1 << 29)
    g = load_golden("beem_c2.json")
    m = synth.beem_shaped_model(**g["model"])
    ctx = cuda_lib.ReachContext(None, 16, max_levels=1 << 14, n_buckets=nb)
    got = ctx.reach(m, mode=cuda_lib.REACH_PERSISTENT)
    assert (got.states, got.transitions, got.deadlocks, got.digest) == (
        g["states"], g["transitions"], g["deadlocks"], int(g["digest"], 16))
    assert got.level_sizes == g["level_sizes"]
    ctx.close()
    del ctx
    torch.cuda.empty_cache()
