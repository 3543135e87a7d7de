"""Closed forms of the interleaving family, for models of any size (test helper).

An interleaving model is P independent processes, each a strongly connected
local automaton; a global step moves one process along one of its edges.  So
(Alg. "Reachability analysis" run from init = 0):

* the reachable set is the whole product space {0..n_0-1} x ... x {0..n_P-1}
  (padding words stay 0), and states = prod n_p;
* every state enables E_p edges of process p whose source is its local state,
  so transitions = sum over p of E_p * prod_{q != p} n_q, with E_p the number
  of edges of automaton p (edges counted with multiplicity);
* no state is a deadlock (every local state has an out-edge);
* the BFS distance of a global state is the sum of its components' distances
  in their automata (a shortest path moves each process independently), so the
  level sizes are the convolution of the automata's BFS layer histograms;
* the set digest is the sum of the oracle's state fingerprint over the product
  space, enumerated here in chunks so that spaces of 10^8 states and more fit
  in memory.

The only arithmetic of the method used here is the oracle's own fingerprint
(oracle.digest); everything else is the mathematics above.
"""
from __future__ import annotations

import math

import numpy as np

import oracle


def local_layers(m, p) -> np.ndarray:
    """BFS layer histogram of process p's automaton from init[p]."""
    n = int(m.n_local[p])
    dist = [-1] * n
    s0 = int(m.init[p])
    dist[s0] = 0
    queue = [s0]
    for s in queue:
        for e in m.edges_of(p, s):
            d = int(m.edge_dst[e])
            if dist[d] < 0:
                dist[d] = dist[s] + 1
                queue.append(d)
    assert min(dist) >= 0, f"{m.name}: automaton {p} is not strongly connected"
    return np.bincount(dist).astype(np.int64)


def is_interleaving(m) -> bool:
    """No shared variables, no guards, no updates, no critical states, init 0."""
    return (m.n_shared == 0 and (m.guard_var < 0).all() and (m.upd_var < 0).all()
            and (m.crit < 0).all() and not np.any(m.init))


def product_digest(m, chunk: int = 1 << 22) -> int:
    """Sum mod 2^64 of the oracle fingerprint over the product space."""
    n = [int(x) for x in m.n_local]
    total = math.prod(n)
    acc = 0
    rows = np.zeros((min(chunk, total), m.state_words), dtype=np.int32)
    for start in range(0, total, chunk):
        k = min(chunk, total - start)
        idx = np.arange(start, start + k, dtype=np.int64)
        blk = rows[:k]
        # mixed radix, last process fastest (any order enumerates the same set)
        for p in range(m.n_procs - 1, -1, -1):
            blk[:, p] = idx % n[p]
            idx //= n[p]
        acc = (acc + oracle.digest(blk)) & ((1 << 64) - 1)
    return acc


def expected(m, chunk: int = 1 << 22) -> dict:
    """states, transitions, deadlocks, level sizes and digest of an
    interleaving model, from the closed forms."""
    assert is_interleaving(m), m.name
    n = [int(x) for x in m.n_local]
    states = math.prod(n)
    base = [int(x) for x in m.local_base]
    E = [int(m.edge_begin[base[p] + n[p]] - m.edge_begin[base[p]]) for p in range(m.n_procs)]
    transitions = sum(E[p] * (states // n[p]) for p in range(m.n_procs))
    levels = np.array([1], dtype=np.int64)
    for p in range(m.n_procs):
        levels = np.convolve(levels, local_layers(m, p))
    assert int(levels.sum()) == states
    return {"states": states, "transitions": transitions, "deadlocks": 0,
            "level_sizes": [int(x) for x in levels], "digest": product_digest(m, chunk)}
