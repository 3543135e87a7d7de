"""The exchange of owner-partitioned reachability between processes (no GPU).

Two gloo ranks each hold successors (seeded int32 rows) with owners; after
paper_1004_2772_gb300.exchange.exchange, each rank must hold exactly the rows
it owns, grouped by source rank in rank order and in the source's order inside
a group, and the count matrix and the offsets of `plan` must describe that
layout -- the same layout the one-GPU partitioned driver builds in its inbox.
Edge cases: a rank that sends nothing to one owner, and a rank with no rows.
"""
import os
import socket

import numpy as np
import pytest

from paper_1004_2772_gb300 import exchange


def _rows(rank, n, w=16):
    rng = np.random.default_rng(1000 + rank)
    rows = rng.integers(-2**31, 2**31 - 1, size=(n, w), dtype=np.int64).astype(np.int32)
    rows[:, 0] = np.arange(n, dtype=np.int32) * 2 + rank   # distinct across ranks
    return rows


def _owners(rows, world, case):
    if case == "one-sided":          # rank 0 sends everything to rank 1
        return np.ones(rows.shape[0], dtype=np.int64) if rows[0, 0] % 2 == 0 else \
            (rows[:, 1].astype(np.int64) & 1)
    return (rows[:, 1].astype(np.int64) & 0x7FFFFFFF) % world


def _inputs(rank, world, case):
    n = {"mixed": (1000, 777), "one-sided": (500, 300), "empty": (0, 400)}[case][rank]
    rows = _rows(rank, n)
    owners = _owners(rows, world, case) if n else np.zeros(0, dtype=np.int64)
    return rows, owners


def _worker(rank, world, port, case, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rows, owners = _inputs(rank, world, case)
        recv, counts = exchange.exchange(torch.from_numpy(rows), torch.from_numpy(owners))
        # what every rank sent, rebuilt locally from the seeds
        expect = [r[o == rank] for r, o in (_inputs(s, world, case) for s in range(world))]
        want_counts = np.array([[int((_inputs(s, world, case)[1] == o).sum()) for o in range(world)]
                                for s in range(world)])
        ok = np.array_equal(counts, want_counts)
        ok &= np.array_equal(recv.numpy(), np.concatenate(expect, axis=0).reshape(-1, 16))
        seg_off, in_begin = exchange.plan(counts)
        # this rank's inbox is owner `rank`'s range of the one-GPU layout
        base = in_begin[rank]
        for s in range(world):
            lo = seg_off[s, rank] - base
            seg = recv.numpy()[lo:lo + counts[s, rank]]
            ok &= np.array_equal(seg, expect[s])
        ok &= int(in_begin[rank + 1] - in_begin[rank]) == recv.shape[0]
        q.put((rank, bool(ok)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("case", ["mixed", "one-sided", "empty"])
def test_two_rank_exchange_gloo(case):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: True, 1: True}


def test_plan_layout():
    c = np.array([[3, 0, 2], [1, 4, 0], [0, 0, 5]])
    seg_off, in_begin = exchange.plan(c)
    assert in_begin.tolist() == [0, 4, 8, 15]
    # owner 0: source 0 (3 rows) then source 1 (1 row); owner 2: sources 0 (2), 2 (5)
    assert seg_off[:, 0].tolist() == [0, 3, 4] and seg_off[:, 2].tolist() == [8, 10, 10]
    assert exchange.rank_splits(c, 1) == ([1, 4, 0], [0, 4, 0])
    z, b = exchange.plan(np.zeros((4, 4), dtype=int))
    assert b.tolist() == [0] * 5 and (z == 0).all()
