"""The exchange step of owner-partitioned reachability between processes.

The partitioned driver (part_reach_* in include/reach.h) keeps K owner
partitions on one GPU, and its exchange is an in-device scatter: the
successors counted per (source partition s, owner o) are placed so that owner
o's inbox holds the segments (0, o), (1, o), ..., (K-1, o) in that order.
With one partition per process, the same step is an all-to-all (the static
partitioning of Sec. 4.1, where every successor goes to the queue of the worker
its hash assigns it to): each rank orders its successors by owner, the
per-owner counts are exchanged first, then the rows, and rank o receives the
segments of every source rank in rank order -- the same layout.

`plan` is that layout from the count matrix (host arithmetic; the device plan
of the one-GPU driver must agree with it), `exchange` the all-to-all over
torch.distributed for one level's successors.  The exchange is tested with the
gloo backend on CPU, two ranks; it has not been run on GPUs.
"""
from __future__ import annotations

import numpy as np


def plan(counts) -> tuple[np.ndarray, np.ndarray]:
    """counts[s, o] = rows from source s owned by o.  Returns (seg_off[s, o],
    in_begin[o], K + 1 entries): owner o's rows start at in_begin[o], and the
    segment from source s at seg_off[s, o] = in_begin[o] + sum of counts[s', o]
    over s' < s."""
    c = np.asarray(counts, dtype=np.int64)
    K = c.shape[0]
    assert c.shape == (K, K) and (c >= 0).all()
    in_begin = np.zeros(K + 1, dtype=np.int64)
    in_begin[1:] = np.cumsum(c.sum(axis=0))
    seg_off = in_begin[:K][None, :] + np.cumsum(c, axis=0) - c
    return seg_off, in_begin


def rank_splits(counts, rank: int) -> tuple[list, list]:
    """all_to_all split sizes of `rank`: rows it sends to each owner (its row
    of counts) and rows it receives from each source (its column)."""
    c = np.asarray(counts, dtype=np.int64)
    return [int(x) for x in c[rank, :]], [int(x) for x in c[:, rank]]


def exchange(rows, owners, group=None):
    """All-to-all of one level's successors.

    rows: [n, w] tensor of this rank's successors; owners: [n] int64 tensor,
    the owner rank of each row.  Returns (received rows: every rank's rows
    owned by this rank, grouped by source rank in rank order and, inside a
    source, in that source's order; counts [world, world] as a numpy array,
    counts[s, o] = rows sent from s to o)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    owners = owners.to(torch.int64)
    if owners.numel() and (int(owners.min()) < 0 or int(owners.max()) >= world):
        raise ValueError("owner outside [0, world)")
    order = torch.argsort(owners, stable=True)
    send = rows[order].contiguous()
    mine = torch.bincount(owners, minlength=world).to(torch.int64)
    # the count matrix first (every rank learns every rank's sends), then the rows
    all_counts = [torch.zeros(world, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_counts, mine, group=group)
    counts = torch.stack(all_counts).numpy()
    send_splits, recv_splits = rank_splits(counts, rank)
    recv = rows.new_empty((sum(recv_splits),) + tuple(rows.shape[1:]))
    dist.all_to_all_single(recv, send, output_split_sizes=recv_splits, input_split_sizes=send_splits,
                           group=group)
    return recv, counts
