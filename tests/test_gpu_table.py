"""find-or-put on the GPU against the oracle (through the C ABI).

Parity bar (integer work): bit-exact.  Which of several equal keys in one
batch is reported new, and which bucket a key lands in, are not unique; the
tests compare what is unique -- for every distinct key exactly one call
answers "new" and it lies in the batch of the key's first occurrence, all
calls of a key get one idx, distinct keys get distinct idx, the stored rows
equal the keys -- and the table-wide invariants: done buckets = distinct keys,
no bucket left in the write state, digest of the stored set = oracle digest.
"""
import numpy as np
import pytest

import oracle
from paper_1004_2772_gb300 import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def run_batches(b, tab, keys, n_batches):
    torch = _torch()
    n = keys.shape[0]
    cuts = np.linspace(0, n, n_batches + 1).astype(np.int64)
    seen, idx = [], []
    for i in range(n_batches):
        k = torch.from_numpy(np.ascontiguousarray(keys[cuts[i]:cuts[i + 1]])).cuda()
        s, x = tab.find_or_put(k)
        seen.append(s)
        idx.append(x)
    torch.cuda.synchronize()
    return (torch.cat(seen).cpu().numpy(), torch.cat(idx).cpu().numpy().view(np.uint32), cuts)


def check_parity(tab, keys, seen, idx, cuts):
    ref = oracle.find_or_put_stream(keys)
    first = ref.first.astype(np.int64)
    assert (seen <= 1).all(), "device error reported"
    # one idx per key, distinct keys -> distinct idx
    assert np.array_equal(idx, idx[first])
    uniq_first = np.unique(first)
    assert np.unique(idx[uniq_first]).shape[0] == uniq_first.shape[0]
    # exactly one 'new' per distinct key, in the batch of its first occurrence
    new_pos = np.nonzero(seen == 0)[0]
    assert new_pos.shape[0] == ref.n_new
    assert np.array_equal(np.sort(first[new_pos]), uniq_first)
    batch_of = np.searchsorted(cuts, np.arange(keys.shape[0]), side="right") - 1
    assert np.array_equal(batch_of[new_pos], batch_of[first[new_pos]])
    # stored rows and table-wide invariants
    torch = _torch()
    got = tab.gather(torch.from_numpy(idx.view(np.int32)).cuda()).cpu().numpy()
    assert np.array_equal(got, keys)
    done, writing, digest = tab.scan()
    assert (done, writing) == (ref.n_new, 0)
    assert digest == ref.digest
    st = tab.stats()
    assert st.stored == ref.n_new and st.error == 0


@pytest.mark.parametrize("W", [1, 5, 8, 16, 32])
@pytest.mark.parametrize("L", [8, 16, 32])
def test_stream_parity_shapes(cuda_lib, W, L):
    rng = np.random.default_rng(W * 100 + L)
    n_ids = 20000
    ids = synth.call_ids(W + L, n_ids, 0, 2 * n_ids, "uniform")
    keys = synth.key_words(W * 7 + L, ids, W)
    perm = rng.permutation(keys.shape[0])      # mix new and repeated keys inside batches
    keys = np.ascontiguousarray(keys[perm])
    tab = cuda_lib.Table(16, W, line_buckets=L)  # load factor ~0.3
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 3)
    check_parity(tab, keys, seen, idx, cuts)
    assert tab.sync() == cuda_lib.HT_OK


@pytest.mark.parametrize("dedup", [0, 1])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_stream_parity_hot_keys(cuda_lib, dedup, dist):
    n_ids = 1 << 15
    zt = synth.zipf_table(n_ids) if dist == "zipf" else None
    ids = synth.call_ids(77, n_ids, 0, 2 * n_ids, dist, zt)
    keys = synth.key_words(78, ids, 16)
    tab = cuda_lib.Table(16, 16, dedup=dedup)  # load factor 0.5
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 4)
    check_parity(tab, keys, seen, idx, cuts)


@pytest.mark.parametrize("lf_log2", [(6, 57), (8, 230), (10, 1000)])
def test_high_load_forces_rehash(cuda_lib, lf_log2):
    """Tiny tables at 90-98% load: long walks, rehash rounds and CAS races."""
    log2, n_ids = lf_log2
    ids = np.repeat(np.arange(n_ids, dtype=np.uint64), 3)
    np.random.default_rng(log2).shuffle(ids)
    keys = synth.key_words(5, ids, 16)
    tab = cuda_lib.Table(log2, 16, line_buckets=8)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 1)
    check_parity(tab, keys, seen, idx, cuts)
    assert tab.stats().rehashes > 0


def test_full_table_reports_full_and_stays_valid(cuda_lib):
    torch = _torch()
    keys = synth.key_words(9, np.arange(40, dtype=np.uint64), 16)
    tab = cuda_lib.Table(4, 16, line_buckets=8)   # 16 buckets, 40 distinct keys
    s, x = tab.find_or_put(torch.from_numpy(keys).cuda())
    torch.cuda.synchronize()
    s = s.cpu().numpy()
    assert tab.sync() == cuda_lib.HT_ERR_FULL
    assert (s == 0).sum() <= 16 and (s == 2).sum() >= 24
    done, writing, _ = tab.scan()
    assert writing == 0 and done == (s == 0).sum() == 16


def test_empty_batch_and_clear(cuda_lib):
    torch = _torch()
    tab = cuda_lib.Table(8, 4)
    s, x = tab.find_or_put(torch.zeros((0, 4), dtype=torch.int32, device="cuda"))
    assert s.numel() == 0
    k = torch.arange(8, dtype=torch.int32, device="cuda").view(2, 4)
    s1, x1 = tab.find_or_put(k)
    tab.clear()
    s2, x2 = tab.find_or_put(k)
    torch.cuda.synchronize()
    assert s1.tolist() == [0, 0] and s2.tolist() == [0, 0]
    assert tab.scan()[0] == 2


def test_same_key_many_lanes(cuda_lib):
    """One key repeated across whole warps: one 'new', everyone the same idx."""
    torch = _torch()
    for dedup in (0, 1):
        tab = cuda_lib.Table(10, 16, dedup=dedup)
        k = torch.full((4096, 16), 7, dtype=torch.int32, device="cuda")
        s, x = tab.find_or_put(k)
        torch.cuda.synchronize()
        assert int((s == 0).sum()) == 1 and int((s == 1).sum()) == 4095
        assert int(x.min()) == int(x.max())


def test_uniform_stream_structure_at_scale(cuda_lib):
    """2^22 buckets at load factor 0.75 (3.1M keys, 6.3M calls).  The uniform
    stream repeats only earlier ids, so each id's calls all share one idx, the
    id's first call (2i) lies in the earliest batch holding any of its calls,
    and exactly one call per id answers new -- properties of the input that
    hold at any size, checked without the oracle's per-call replay."""
    torch = _torch()
    log2 = 22
    n_ids = (3 << log2) // 4
    ids = synth.call_ids(123, n_ids, 0, 2 * n_ids, "uniform")
    keys = synth.key_words(124, ids, 16)
    tab = cuda_lib.Table(log2, 16)
    seen, idx, cuts = run_batches(cuda_lib, tab, keys, 2)
    assert (seen <= 1).all()
    ids = ids.astype(np.int64)
    assert np.array_equal(np.bincount(ids[seen == 0], minlength=n_ids), np.ones(n_ids, np.int64))
    assert np.array_equal(idx, idx[2 * ids])
    assert np.unique(idx[0::2]).shape[0] == n_ids
    batch_of = np.searchsorted(cuts, np.arange(ids.shape[0]), side="right") - 1
    new_pos = np.nonzero(seen == 0)[0]
    assert np.array_equal(batch_of[new_pos], batch_of[2 * ids[new_pos]])
    done, writing, digest = tab.scan()
    assert (done, writing) == (n_ids, 0)
    assert digest == oracle.digest(synth.key_words(124, np.arange(n_ids, dtype=np.uint64), 16))
