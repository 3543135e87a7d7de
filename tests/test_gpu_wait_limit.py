"""The bounded wait on a write-busy bucket (Sec. 3, Alg. "find-or-put": a
bucket whose memo matches but whose data is still being written is polled
until its writer publishes it).

The wait must end even when no writer ever publishes: a bucket is planted in
the write state (its done bit cleared on the device, the memo kept), so the
next find-or-put of its key polls a flag that nothing sets.  After max_spin
polls the kernel latches HT_ERR_TIMEOUT, reports the call as an error and
returns; the other calls of the batch are answered, and the table stays
usable: publishing the bucket again makes the key findable, and a clear
resets the error.  Nothing here faults or hangs the GPU: each poll is a load
of a bucket inside the table, and the number of polls is bounded.
"""
import numpy as np
import pytest

from paper_1004_2772_gb300 import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("bucket_bits,group_lanes", [(32, 1), (16, 1), (32, 4)])
def test_unpublished_bucket_times_out_and_table_stays_usable(cuda_lib, bucket_bits, group_lanes):
    torch = _torch()
    params = dict(max_spin=64, bucket_bits=bucket_bits)
    if group_lanes > 1:
        params.update(group_lanes=group_lanes, line_buckets=4 * group_lanes)
    tab = cuda_lib.Table(12, 16, **params)
    keys = torch.from_numpy(synth.key_words(11, np.arange(64, dtype=np.uint64), 16)).cuda()
    s, x = tab.find_or_put(keys)
    torch.cuda.synchronize()
    assert tab.sync() == cuda_lib.HT_OK
    assert (s.cpu().numpy() == 0).all()
    idx = x.cpu().numpy().view(np.uint32)

    # plant: key 5's bucket back in the write state (done bit cleared, memo kept)
    buckets, _ = tab.arrays()
    i = int(idx[5])
    done_mask = 0x7FFFFFFF if bucket_bits == 32 else 0x7FFF
    before = int(buckets[i].item())
    assert before & ~done_mask, "a stored key's bucket has its done bit set"
    buckets[i] = before & done_mask
    torch.cuda.synchronize()
    assert tab.scan()[1] == 1  # one bucket in the write state

    s2, x2 = tab.find_or_put(keys)
    torch.cuda.synchronize()
    s2 = s2.cpu().numpy()
    assert tab.sync() == cuda_lib.HT_ERR_TIMEOUT
    assert s2[5] == 2, "the call that waited on the unpublished bucket reports an error"
    others = np.arange(64) != 5
    assert (s2[others] == 1).all(), "every other key is still found"
    assert np.array_equal(x2.cpu().numpy().view(np.uint32)[others], idx[others])
    st = tab.stats()
    assert st.busy_waits >= 1 and st.error == cuda_lib.HT_ERR_TIMEOUT

    # publish the bucket again: the key is found where it was stored
    buckets[i] = before
    torch.cuda.synchronize()
    s3, x3 = tab.find_or_put(keys[5:6].contiguous())
    torch.cuda.synchronize()
    assert s3.cpu().tolist() == [1] and int(x3.cpu().numpy().view(np.uint32)[0]) == i
    assert tab.scan()[:2] == (64, 0)

    # a clear resets the error word; the table works as new
    tab.clear()
    assert tab.sync() == cuda_lib.HT_OK
    s4, _ = tab.find_or_put(keys)
    torch.cuda.synchronize()
    assert (s4.cpu().numpy() == 0).all() and tab.sync() == cuda_lib.HT_OK
    tab.close()
